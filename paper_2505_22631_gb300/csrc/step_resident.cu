// step_resident.cu -- the resident form: one launch runs every step.
//
// Replicas are independent trajectories, so a thread block that owns a group of
// whole replicas of one graph can run all T steps of Algorithm 1 with only
// block-level barriers: there is no grid-wide synchronisation at all.  The
// block keeps the (cos, sin) cache of all n nodes of its replicas in shared
// memory, which is what every neighbour gather reads.  A phase is read only by
// the thread that owns it, so phases stay in the [node][R_pad] device array
// (read and written once per step, coalesced, L2-resident for the workloads
// here); the CSR structure is read through the read-only cache.
//
// Thread layout inside a block: thread = (node slot, replica unit u), u fastest,
// where a unit is U = 2 replicas (U = 1 when a graph is too large for two).
// A thread owns nodes slot, slot + NS, slot + 2 NS, ... (NS = threads / units).
// One step:
//   phase A: gather (A, B) = sum_j w_ij (c_j, s_j) from shared memory, draw the
//            noise, write the new phases (old cache only: synchronous update)
//   barrier
//   phase B: write the new (cos, sin) of owned nodes into the cache
//   barrier
// Every readout step the block thresholds its phases, writes the spins of its
// replicas to device memory and sums the agreeing weight of each replica.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {

namespace {

// (cos, sin) of one replica in shared memory: FP32, FP16 or BF16 pairs.
struct CacheF32 {
    using T = float2;
    __device__ static T pack(float2 cs) { return cs; }
    __device__ static float2 unpack(const T& v) { return v; }
};
struct CacheF16 {
    using T = __half2;
    __device__ static T pack(float2 cs) { return __floats2half2_rn(cs.x, cs.y); }
    __device__ static float2 unpack(const T& v) { return __half22float2(v); }
};
struct CacheBF16 {
    using T = __nv_bfloat162;
    __device__ static T pack(float2 cs) { return __floats2bfloat162_rn(cs.x, cs.y); }
    __device__ static float2 unpack(const T& v) { return __bfloat1622float2(v); }
};

__device__ __forceinline__ float2 cos_sin_2pi(float th) {
    float s, c;
    sincospif(2.0f * th, &s, &c);
    return make_float2(c, s);
}

template <int U, typename T>
struct Unit;   // U consecutive cache entries loaded together
template <typename T>
struct Unit<1, T> { T v[1]; };
template <typename T>
struct __align__(2 * sizeof(T)) Unit<2, T> { T v[2]; };

struct ResidentArgs {
    CSRDev csr;
    StepParams P;
    const int4* items;      // per block: (graph, first replica, replicas in group, 0)
    float* theta;           // [nodes][R_pad], the phases, updated in place
    int8_t* spins;          // [nodes][R_pad] readout scratch
    double* agree;          // [G][row_stride][R_pad]
    int64_t row_stride;
    int64_t readout_every;
};

template <int U>
__device__ __forceinline__ void load_theta(const float* p, float (&th)[U]) {
    if (U == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        th[0] = v.x;
        th[U - 1] = v.y;
    } else {
        th[0] = *p;
    }
}

template <int U>
__device__ __forceinline__ void store_theta(float* p, const float (&th)[U]) {
    if (U == 2)
        *reinterpret_cast<float2*>(p) = make_float2(th[0], th[U - 1]);
    else
        *p = th[0];
}

// Normals of replicas r .. r+U-1 (r even when U == 2) at step t.
template <int U>
__device__ __forceinline__ void noise_unit(uint64_t seed, uint32_t g, uint32_t i, uint32_t t,
                                           uint32_t r, float (&z)[U]) {
    const uint4 x = draw_block(seed, g, kStreamNoise, i, t, r >> 2);
    const float2 zz = (r & 2) ? box_muller(x.z, x.w) : box_muller(x.x, x.y);
    if (U == 2) {
        z[0] = zz.x;
        z[U - 1] = zz.y;
    } else {
        z[0] = (r & 1) ? zz.y : zz.x;
    }
}

template <int U>
__device__ __forceinline__ void init_unit(uint64_t seed, uint32_t g, uint32_t i, uint32_t r,
                                          float (&th)[U]) {
    const uint4 x = draw_block(seed, g, kStreamInit, i, 0, r >> 2);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int u = 0; u < U; ++u) th[u] = u01(w[(r + u) & 3]);
}

template <int U, bool kUnit, typename Cache>
__global__ void __launch_bounds__(1024, 1) resident_kernel(ResidentArgs a) {
    using T = typename Cache::T;
    using UT = Unit<U, T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    UT* cache = reinterpret_cast<UT*>(smem_raw);   // [n][units]

    const int4 item = a.items[blockIdx.x];
    const int g = item.x, r0 = item.y, kk = item.z;
    const GraphDev gd = a.csr.graphs[g];
    const int n = gd.n, noff = gd.node_off;
    const int units = kk / U;
    const int NS = blockDim.x / units;
    const int u = threadIdx.x % units;
    const int slot = threadIdx.x / units;
    const int i_begin = slot < NS ? slot : n;   // idle threads own no node
    const int r = r0 + U * u;
    const StepParams& P = a.P;
    const int R_pad = P.R_pad;
    float* theta = a.theta + r;                   // theta[node * R_pad] of this unit

    for (int i = i_begin; i < n; i += NS) {
        float th[U];
        init_unit<U>(P.seed, (uint32_t)g, (uint32_t)i, (uint32_t)r, th);
        store_theta<U>(theta + (size_t)(noff + i) * R_pad, th);
        UT c;
#pragma unroll
        for (int v = 0; v < U; ++v) c.v[v] = Cache::pack(cos_sin_2pi(th[v]));
        cache[i * units + u] = c;
    }
    __syncthreads();

    const float sdt = P.sqrt_dt;
    const size_t sbase = (size_t)g * P.steps;
    int64_t next_readout = a.readout_every > 0 ? a.readout_every : -1;
    for (int64_t t = 0; t < P.steps; ++t) {
        const float K = __ldg(P.K + sbase + t), Ks = __ldg(P.Ks + sbase + t);
        const float Kn = __ldg(P.Kn + sbase + t);
        const float dtK = P.dt * K, dtKs = P.dt * Ks, kick = Kn * sdt;
        for (int i = i_begin; i < n; i += NS) {
            const int node = noff + i;
            float th[U];
            load_theta<U>(theta + (size_t)node * R_pad, th);
            const UT own = cache[i * units + u];
            float2 acc[U];
#pragma unroll
            for (int v = 0; v < U; ++v) acc[v] = make_float2(0.f, 0.f);
            const int e_end = __ldg(a.csr.rowp + node + 1);
#pragma unroll 4
            for (int e = __ldg(a.csr.rowp + node); e < e_end; ++e) {
                const uint32_t cw = __ldg(a.csr.col + e);
                float w;
                int jj;
                if (kUnit) {
                    jj = (int)(cw & ~kSignBit) - noff;
                    w = (cw & kSignBit) ? -1.0f : 1.0f;
                } else {
                    jj = (int)cw - noff;
                    w = __ldg(a.csr.w + e);
                }
                const UT nb = cache[jj * units + u];
                const float2 ww = make_float2(w, w);
#pragma unroll
                for (int v = 0; v < U; ++v) acc[v] = ffma2(Cache::unpack(nb.v[v]), ww, acc[v]);
            }
            float z[U];
            noise_unit<U>(P.seed, (uint32_t)g, (uint32_t)i, (uint32_t)t, (uint32_t)r, z);
#pragma unroll
            for (int v = 0; v < U; ++v) {
                const float2 o = Cache::unpack(own.v[v]);
                const float d = o.y * acc[v].x - o.x * acc[v].y;
                th[v] = wrap01(th[v] + (dtK * d - dtKs * sin_q(P.q, o.x, o.y)) + kick * z[v]);
            }
            store_theta<U>(theta + (size_t)node * R_pad, th);
        }
        __syncthreads();
        for (int i = i_begin; i < n; i += NS) {
            float th[U];
            load_theta<U>(theta + (size_t)(noff + i) * R_pad, th);
            UT c;
#pragma unroll
            for (int v = 0; v < U; ++v) c.v[v] = Cache::pack(cos_sin_2pi(th[v]));
            cache[i * units + u] = c;
        }
        __syncthreads();

        if (t + 1 == next_readout) {
            const int64_t k = next_readout / a.readout_every - 1;
            next_readout += a.readout_every;
            if (threadIdx.x < kk) red[threadIdx.x] = 0.0;
            for (int i = i_begin; i < n; i += NS) {
                float th[U];
                load_theta<U>(theta + (size_t)(noff + i) * R_pad, th);
#pragma unroll
                for (int v = 0; v < U; ++v)
                    a.spins[(size_t)(noff + i) * R_pad + r + v] = (int8_t)spin_of(th[v], P.q);
            }
            __syncthreads();
            float f[U];
#pragma unroll
            for (int v = 0; v < U; ++v) f[v] = 0.f;
            for (int i = i_begin; i < n; i += NS) {
                const int node = noff + i;
                int8_t si[U];
#pragma unroll
                for (int v = 0; v < U; ++v) si[v] = a.spins[(size_t)node * R_pad + r + v];
                const int e_end = a.csr.rowp[node + 1];
                for (int e = a.csr.rowp[node]; e < e_end; ++e) {
                    const uint32_t cw = a.csr.col[e];
                    const int jn = kUnit ? (int)(cw & ~kSignBit) : (int)cw;
                    if (jn <= node) continue;
                    const float w = kUnit ? ((cw & kSignBit) ? -1.0f : 1.0f) : a.csr.w[e];
#pragma unroll
                    for (int v = 0; v < U; ++v)
                        f[v] += (si[v] == a.spins[(size_t)jn * R_pad + r + v]) ? w : 0.f;
                }
            }
            if (slot < NS) {
#pragma unroll
                for (int v = 0; v < U; ++v)
                    if (f[v] != 0.f) atomicAdd(&red[U * u + v], (double)f[v]);
            }
            __syncthreads();
            if (threadIdx.x < kk)
                a.agree[((int64_t)g * a.row_stride + k) * R_pad + r0 + threadIdx.x] = red[threadIdx.x];
        }
    }
}

template <int U, bool kUnit, typename Cache>
cudaError_t launch_one(const ResidentArgs& a, int blocks, int threads, size_t smem, cudaStream_t s) {
    auto fn = resident_kernel<U, kUnit, Cache>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename Cache>
cudaError_t launch_u(int U, bool unit, const ResidentArgs& a, int blocks, int threads, size_t smem,
                     cudaStream_t s) {
    if (U == 2)
        return unit ? launch_one<2, true, Cache>(a, blocks, threads, smem, s)
                    : launch_one<2, false, Cache>(a, blocks, threads, smem, s);
    return unit ? launch_one<1, true, Cache>(a, blocks, threads, smem, s)
                : launch_one<1, false, Cache>(a, blocks, threads, smem, s);
}

}  // namespace

size_t resident_cache_bytes(int32_t prec) { return prec == OIM_PREC_FP32 ? 8 : 4; }

constexpr size_t kSmemBudget = 227 * 1024 - 1024;

// Shape of a resident launch: replicas per block k (at most 64; even unless a
// single replica is all that fits), threads and dynamic shared memory.  Fails
// when not even one replica of the largest graph fits in shared memory.
cudaError_t resident_shape(const oim_problem_s& p, int32_t R_pad, int32_t prec, int32_t want_k,
                           int32_t want_threads, int32_t* k_out, int32_t* threads_out,
                           int32_t* items_out, size_t* smem_out) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t rep_bytes = resident_cache_bytes(prec) * (size_t)p.max_n;
    int k_fit = (int)std::min<size_t>(64, kSmemBudget / rep_bytes);
    if (k_fit >= 2) k_fit &= ~1;
    if (k_fit < 1) return cudaErrorInvalidValue;
    int k;
    if (want_k > 0) {
        k = want_k;
        if (k > k_fit || (k > 1 && (k & 1))) return cudaErrorInvalidValue;
    } else {
        // enough blocks to give every SM one, as few replicas per block as that allows
        const int64_t total = (int64_t)p.G * R_pad;
        const int64_t per = (total + sms - 1) / sms;
        k = (int)std::min<int64_t>(k_fit, std::max<int64_t>(1, per));
        if (k > 1) k = std::min(k_fit, (k + 1) & ~1);
    }
    k = std::min(k, R_pad);
    const int U = (k % 2 == 0) ? 2 : 1;
    const int units = k / U;
    int threads = want_threads > 0 ? want_threads : 1024;
    threads = std::min(1024, std::max(threads, 32 * ((units + 31) / 32)));
    // no more threads than (node, unit) items of the largest graph
    const int64_t work = (int64_t)p.max_n * units;
    if (want_threads <= 0 && work < threads) threads = std::max(32, (int)((work + 31) / 32) * 32);
    int items = 0;
    for (int g = 0; g < p.G; ++g) items += (R_pad + k - 1) / k;
    *k_out = k;
    *threads_out = threads;
    *items_out = items;
    *smem_out = rep_bytes * (size_t)k;
    return cudaSuccess;
}

StepParams make_params(const oim_run_s& r);

cudaError_t launch_resident_impl(const oim_run_s& r, const int4* d_items, cudaStream_t s) {
    ResidentArgs a;
    a.csr = r.p->csr();
    a.P = make_params(r);
    a.items = d_items;
    a.theta = r.d_theta[0];
    a.spins = r.d_spins;
    a.agree = r.d_trace;
    a.row_stride = r.readouts_cap;
    a.readout_every = r.readout_every;
    const int U = (r.res_k % 2 == 0) ? 2 : 1;
    const bool unit = r.p->unit_weights;
    if (r.prec == OIM_PREC_FP32)
        return launch_u<CacheF32>(U, unit, a, r.res_items, r.res_threads, r.res_smem, s);
    if (r.prec == OIM_PREC_FP16)
        return launch_u<CacheF16>(U, unit, a, r.res_items, r.res_threads, r.res_smem, s);
    return launch_u<CacheBF16>(U, unit, a, r.res_items, r.res_threads, r.res_smem, s);
}

}  // namespace oim

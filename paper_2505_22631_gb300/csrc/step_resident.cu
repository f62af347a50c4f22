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

#include "oim_checks.cuh"
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
    int64_t T;              // steps to run (P.steps is the schedules' row stride, which a
                            // re-run with fewer steps leaves larger)
    int32_t double_buffer;  // quad kernel: ping-pong (cos, sin) caches in shared memory
    int32_t integer_weights;   // scores accumulate exactly in 32-bit integers
};

// Block-level accumulation of the agreeing weight of each replica at a readout:
// native 32-bit shared-memory atomics (integers when every weight is an integer,
// exact; FP32 otherwise), written out as FP64.
struct ReadoutAcc {
    int32_t i[64];
    float f[64];
};
__device__ __forceinline__ void acc_clear(ReadoutAcc& r, int slot) {
    r.i[slot] = 0;
    r.f[slot] = 0.f;
}
__device__ __forceinline__ void acc_add(ReadoutAcc& r, int slot, float v, bool integer) {
    if (integer)
        atomicAdd(&r.i[slot], __float2int_rn(v));
    else
        atomicAdd(&r.f[slot], v);
}
__device__ __forceinline__ double acc_get(const ReadoutAcc& r, int slot, bool integer) {
    return integer ? (double)r.i[slot] : (double)r.f[slot];
}

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
    __shared__ ReadoutAcc red;
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
    for (int64_t t = 0; t < a.T; ++t) {
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
                jj = checked_local(a.csr, n, jj, i);
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
            if (threadIdx.x < kk) acc_clear(red, threadIdx.x);
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
                    const int jn = noff + checked_local(a.csr, n, (kUnit ? (int)(cw & ~kSignBit) : (int)cw) - noff, i);
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
                    if (f[v] != 0.f) acc_add(red, U * u + v, f[v], a.integer_weights);
            }
            __syncthreads();
            if (threadIdx.x < kk)
                a.agree[((int64_t)g * a.row_stride + k) * R_pad + r0 + threadIdx.x] = acc_get(red, threadIdx.x, a.integer_weights);
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


// ---------------------------------------------------------------------------
// Quad kernel: a thread owns one node and a quad of four replicas (one Philox
// block per node and step, one CSR read per four replicas).  When the graph's
// structure fits, it is copied once into shared memory as 16-bit local column
// indices with the sign of the +-1 weight in the top bit, so a step never
// leaves the SM except for the owned phases.
// ---------------------------------------------------------------------------
// Transcendentals of a step: accurate library functions with the FP32 cache,
// hardware approximations with a 16-bit cache (whose rounding, 2^-12, is far
// above the approximations' ~1e-6).
struct MathAccurate {
    __device__ static float2 cs(float th) { return cos_sin_2pi(th); }
    __device__ static float2 bm(uint32_t a, uint32_t b) { return box_muller(a, b); }
};
struct MathFast {
    __device__ static float2 cs(float th) { return cos_sin_2pi_fast(th); }
    __device__ static float2 bm(uint32_t a, uint32_t b) { return box_muller_fast(a, b); }
};


struct QuadF32 {
    using Math = MathAccurate;
    struct __align__(16) T { float4 lo, hi; };   // (c0, s0, c1, s1), (c2, s2, c3, s3)
    __device__ static T pack(const float2 (&cs)[4]) {
        return T{make_float4(cs[0].x, cs[0].y, cs[1].x, cs[1].y),
                 make_float4(cs[2].x, cs[2].y, cs[3].x, cs[3].y)};
    }
    __device__ static void unpack(const T& v, float2 (&cs)[4]) {
        cs[0] = make_float2(v.lo.x, v.lo.y);
        cs[1] = make_float2(v.lo.z, v.lo.w);
        cs[2] = make_float2(v.hi.x, v.hi.y);
        cs[3] = make_float2(v.hi.z, v.hi.w);
    }
    // acc[v] += (c_v, s_v)
    __device__ static void accumulate(float2 (&acc)[4], const T& v) {
        acc[0] = __fadd2_rn(acc[0], make_float2(v.lo.x, v.lo.y));
        acc[1] = __fadd2_rn(acc[1], make_float2(v.lo.z, v.lo.w));
        acc[2] = __fadd2_rn(acc[2], make_float2(v.hi.x, v.hi.y));
        acc[3] = __fadd2_rn(acc[3], make_float2(v.hi.z, v.hi.w));
    }
};
// acc += (lo, hi) of a packed 16-bit pair, each half widened inside the add
// (PTX mixed-precision add: f32 = f16 + f32, exact widening, one rounding).

template <typename H2, typename Cvt>
struct QuadHalf {
    using Math = MathFast;
    using T = uint4;   // four 16-bit (c, s) pairs
    __device__ static T pack(const float2 (&cs)[4]) {
        uint32_t w[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            H2 h = Cvt::to(cs[v]);
            w[v] = *reinterpret_cast<uint32_t*>(&h);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static void unpack(const T& q, float2 (&cs)[4]) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int v = 0; v < 4; ++v) cs[v] = Cvt::from(*reinterpret_cast<const H2*>(&w[v]));
    }
    __device__ static void accumulate(float2 (&acc)[4], const T& q) {
        Cvt::add(acc[0], q.x);
        Cvt::add(acc[1], q.y);
        Cvt::add(acc[2], q.z);
        Cvt::add(acc[3], q.w);
    }
};
struct CvtF16 {
    __device__ static __half2 to(float2 x) { return __floats2half2_rn(x.x, x.y); }
    __device__ static float2 from(__half2 h) { return __half22float2(h); }
    __device__ static void add(float2& acc, uint32_t h2) { add_f16x2(acc, h2); }
};
struct CvtBF16 {
    __device__ static __nv_bfloat162 to(float2 x) { return __floats2bfloat162_rn(x.x, x.y); }
    __device__ static float2 from(__nv_bfloat162 h) { return __bfloat1622float2(h); }
    __device__ static void add(float2& acc, uint32_t h2) { add_bf16x2(acc, h2); }
};
using QuadF16 = QuadHalf<__half2, CvtF16>;
using QuadBF16 = QuadHalf<__nv_bfloat162, CvtBF16>;

constexpr uint16_t kLocalSign = 0x8000u;


__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename Quad, bool kSmemCSR, bool kUnit>
__global__ void __launch_bounds__(1024, 1) resident_quad_kernel(ResidentArgs a) {
    using T = typename Quad::T;
    using M = typename Quad::Math;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ReadoutAcc red;

    const int4 item = a.items[blockIdx.x];
    const int g = item.x, r0 = item.y, kk = item.z;
    const GraphDev gd = a.csr.graphs[g];
    const int n = gd.n, noff = gd.node_off, e0 = gd.edge_off;
    const int units = kk >> 2;
    const int NS = blockDim.x / units;
    const int u = threadIdx.x % units;
    const int slot = threadIdx.x / units;
    const int i_begin = slot < NS ? slot : n;
    const int rq = (r0 >> 2) + u;               // replica quad index
    const StepParams& P = a.P;
    const int R_pad = P.R_pad;
    float* theta = a.theta + r0 + 4 * u;

    // [n][units] (cos, sin) cache; with double buffering a second one follows, the
    // steps read one and write the other, and one barrier a step separates them
    const bool db = a.double_buffer != 0;
    const size_t cache_bytes = align16((size_t)n * units * sizeof(T));
    T* cache = reinterpret_cast<T*>(smem_raw);
    T* cache_next = db ? reinterpret_cast<T*>(smem_raw + cache_bytes) : cache;
    int32_t* s_rowp = reinterpret_cast<int32_t*>(smem_raw + (db ? 2 : 1) * cache_bytes);
    int32_t* s_split = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(s_rowp) +
                                                  align16((size_t)(n + 1) * 4));
    uint16_t* s_order = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(s_split) +
                                                    align16((size_t)n * 4));
    uint16_t* s_col = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(s_order) +
                                                  align16((size_t)n * 2));
    if (kSmemCSR) {
        for (int i = threadIdx.x; i <= n; i += blockDim.x) s_rowp[i] = a.csr.rowp[noff + i] - e0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            s_split[i] = a.csr.split[noff + i] - e0;
            s_order[i] = (uint16_t)a.csr.order[noff + i];
        }
        const int nnz_g = a.csr.rowp[noff + n] - e0;
        for (int e = threadIdx.x; e < nnz_g; e += blockDim.x) {
            const uint32_t cw = a.csr.col[e0 + e];
            // (checked builds: a column outside the graph becomes its first node)
            const uint32_t jl = (uint32_t)checked_local(a.csr, n, (int)((cw & ~kSignBit) - (uint32_t)noff), 0);
            s_col[e] = (uint16_t)(jl | ((cw & kSignBit) ? kLocalSign : 0u));
        }
    }
    for (int i = i_begin; i < n; i += NS) {
        const uint4 x = draw_block(P.seed, (uint32_t)g, kStreamInit, (uint32_t)i, 0, (uint32_t)rq);
        const float4 th = make_float4(u01(x.x), u01(x.y), u01(x.z), u01(x.w));
        *reinterpret_cast<float4*>(theta + (size_t)(noff + i) * R_pad) = th;
        const float2 cs[4] = {M::cs(th.x), M::cs(th.y), M::cs(th.z), M::cs(th.w)};
        cache[i * units + u] = Quad::pack(cs);
    }
    __syncthreads();

    const float sdt = P.sqrt_dt;
    const size_t sbase = (size_t)g * P.steps;
    int64_t next_readout = a.readout_every > 0 ? a.readout_every : -1;
    // with double buffering and at most one node a thread, the thread keeps its node's
    // phases in registers and stores them only where a readout or the end reads them
    const bool own1 = db && n <= NS;
    float4 th_keep = make_float4(0.f, 0.f, 0.f, 0.f);
    if (own1 && i_begin < n) {
        const int i0 = kSmemCSR ? (int)s_order[i_begin] : a.csr.order[noff + i_begin];
        th_keep = *reinterpret_cast<const float4*>(theta + (size_t)(noff + i0) * R_pad);
    }
    for (int64_t t = 0; t < a.T; ++t) {
        const float K = __ldg(P.K + sbase + t), Ks = __ldg(P.Ks + sbase + t);
        const float Kn = __ldg(P.Kn + sbase + t);
        const float dtK = P.dt * K, dtKs = P.dt * Ks, kick = Kn * sdt;
        const bool store_theta = !own1 || t + 1 == next_readout || t + 1 == a.T;
        // nodes in order of degree, so the lanes of a warp run rows of equal length;
        // the next node's phases are loaded while the current one is processed
        int i_cur = i_begin < n ? (kSmemCSR ? (int)s_order[i_begin] : a.csr.order[noff + i_begin]) : 0;
        float4 th_cur = own1 ? th_keep
                             : (i_begin < n ? *reinterpret_cast<const float4*>(theta + (size_t)(noff + i_cur) * R_pad)
                                            : make_float4(0.f, 0.f, 0.f, 0.f));
        for (int slot_i = i_begin; slot_i < n; slot_i += NS) {
            const int i = i_cur;
            const float4 th = th_cur;
            const int slot_n = slot_i + NS;
            if (slot_n < n) {
                i_cur = kSmemCSR ? (int)s_order[slot_n] : a.csr.order[noff + slot_n];
                th_cur = *reinterpret_cast<const float4*>(theta + (size_t)(noff + i_cur) * R_pad);
            }
            const int node = noff + i;
            float2 own[4];
            Quad::unpack(cache[i * units + u], own);
            float2 acc[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[v] = make_float2(0.f, 0.f);
            if (kSmemCSR) {
                // rows hold the +1 entries first, then the -1 entries
                const int eb = s_rowp[i], es = s_split[i], ee = s_rowp[i + 1];
                const T* row = cache + u;
#pragma unroll 4
                for (int e = eb; e < es; ++e)
                    Quad::accumulate(acc, row[(s_col[e] & 0x7FFFu) * units]);
                if (es < ee) {   // -1 entries: -( -acc + sum )
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[v] = make_float2(-acc[v].x, -acc[v].y);
#pragma unroll 4
                    for (int e = es; e < ee; ++e)
                        Quad::accumulate(acc, row[(s_col[e] & 0x7FFFu) * units]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[v] = make_float2(-acc[v].x, -acc[v].y);
                }
            } else {
                const int ee = __ldg(a.csr.rowp + node + 1);
                for (int e = __ldg(a.csr.rowp + node); e < ee; ++e) {
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
                    jj = checked_local(a.csr, n, jj, i);
                    float2 nb[4];
                    Quad::unpack(cache[jj * units + u], nb);
                    const float2 ww = make_float2(w, w);
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[v] = ffma2(nb[v], ww, acc[v]);
                }
            }
            const uint4 x = draw_block(P.seed, (uint32_t)g, kStreamNoise, (uint32_t)i, (uint32_t)t,
                                       (uint32_t)rq);
            const float2 z01 = M::bm(x.x, x.y);
            const float2 z23 = M::bm(x.z, x.w);
            const float z[4] = {z01.x, z01.y, z23.x, z23.y};
            const float t0[4] = {th.x, th.y, th.z, th.w};
            float tn[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float d = own[v].y * acc[v].x - own[v].x * acc[v].y;
                tn[v] = wrap01(t0[v] + (dtK * d - dtKs * sin_q(P.q, own[v].x, own[v].y)) + kick * z[v]);
            }
            if (store_theta)
                *reinterpret_cast<float4*>(theta + (size_t)node * R_pad) = make_float4(tn[0], tn[1], tn[2], tn[3]);
            if (db) {
                // the next step's cache, written while this one is still read
                const float2 cs[4] = {M::cs(tn[0]), M::cs(tn[1]), M::cs(tn[2]), M::cs(tn[3])};
                cache_next[i * units + u] = Quad::pack(cs);
            }
            if (own1) th_keep = make_float4(tn[0], tn[1], tn[2], tn[3]);
        }
        __syncthreads();
        if (db) {
            T* tmp = cache;
            cache = cache_next;
            cache_next = tmp;
        } else {
            float4 th_n = i_begin < n ? *reinterpret_cast<const float4*>(theta + (size_t)(noff + i_begin) * R_pad)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = i_begin; i < n; i += NS) {
                const float4 th = th_n;
                if (i + NS < n) th_n = *reinterpret_cast<const float4*>(theta + (size_t)(noff + i + NS) * R_pad);
                const float2 cs[4] = {M::cs(th.x), M::cs(th.y), M::cs(th.z), M::cs(th.w)};
                cache[i * units + u] = Quad::pack(cs);
            }
            __syncthreads();
        }

        if (t + 1 == next_readout) {
            const int64_t k = next_readout / a.readout_every - 1;
            next_readout += a.readout_every;
            if (threadIdx.x < kk) acc_clear(red, threadIdx.x);
            for (int i = i_begin; i < n; i += NS) {
                const float4 th = *reinterpret_cast<const float4*>(theta + (size_t)(noff + i) * R_pad);
                char4 sp;
                sp.x = (char)spin_of(th.x, P.q);
                sp.y = (char)spin_of(th.y, P.q);
                sp.z = (char)spin_of(th.z, P.q);
                sp.w = (char)spin_of(th.w, P.q);
                *reinterpret_cast<char4*>(a.spins + (size_t)(noff + i) * R_pad + r0 + 4 * u) = sp;
            }
            __syncthreads();
            float f[4] = {0.f, 0.f, 0.f, 0.f};
            for (int i = i_begin; i < n; i += NS) {
                const int node = noff + i;
                const char4 si = *reinterpret_cast<const char4*>(a.spins + (size_t)node * R_pad + r0 + 4 * u);
                const int eb = kSmemCSR ? s_rowp[i] : a.csr.rowp[node] - e0;
                const int ee = kSmemCSR ? s_rowp[i + 1] : a.csr.rowp[node + 1] - e0;
                for (int e = eb; e < ee; ++e) {
                    int jl;
                    float w;
                    if (kSmemCSR) {
                        const uint32_t c = s_col[e];
                        jl = (int)(c & 0x7FFFu);
                        w = (c & kLocalSign) ? -1.0f : 1.0f;
                    } else {
                        const uint32_t cw = a.csr.col[e0 + e];
                        jl = checked_local(a.csr, n, (int)(kUnit ? (cw & ~kSignBit) : cw) - noff, i);
                        w = kUnit ? ((cw & kSignBit) ? -1.0f : 1.0f) : a.csr.w[e0 + e];
                    }
                    if (jl <= i) continue;
                    const char4 sj = *reinterpret_cast<const char4*>(a.spins + (size_t)(noff + jl) * R_pad + r0 + 4 * u);
                    f[0] += (si.x == sj.x) ? w : 0.f;
                    f[1] += (si.y == sj.y) ? w : 0.f;
                    f[2] += (si.z == sj.z) ? w : 0.f;
                    f[3] += (si.w == sj.w) ? w : 0.f;
                }
            }
            if ((units & (units - 1)) == 0 && units <= 32) {
                // lanes lane ^ m (m >= units) hold the same replicas: reduce before the atomics
                // (idle lanes carry zeros; integer-valued sums stay exact in FP32 up to 2^24)
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1)
                    if (m >= units)
#pragma unroll
                        for (int v = 0; v < 4; ++v) f[v] += __shfl_xor_sync(0xffffffffu, f[v], m);
                if ((threadIdx.x & 31) < units && slot < NS) {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (f[v] != 0.f) acc_add(red, 4 * u + v, f[v], a.integer_weights);
                }
            } else if (slot < NS) {
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (f[v] != 0.f) acc_add(red, 4 * u + v, f[v], a.integer_weights);
            }
            __syncthreads();
            if (threadIdx.x < kk)
                a.agree[((int64_t)g * a.row_stride + k) * R_pad + r0 + threadIdx.x] = acc_get(red, threadIdx.x, a.integer_weights);
        }
    }
}

template <typename Quad, bool kSmemCSR, bool kUnit>
cudaError_t launch_quad(const ResidentArgs& a, int blocks, int threads, size_t smem, cudaStream_t s) {
    auto fn = resident_quad_kernel<Quad, kSmemCSR, kUnit>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename Quad>
cudaError_t launch_quad_v(bool smem_csr, bool unit, const ResidentArgs& a, int blocks, int threads,
                          size_t smem, cudaStream_t s) {
    if (smem_csr) return launch_quad<Quad, true, true>(a, blocks, threads, smem, s);
    return unit ? launch_quad<Quad, false, true>(a, blocks, threads, smem, s)
                : launch_quad<Quad, false, false>(a, blocks, threads, smem, s);
}

}  // namespace

size_t resident_cache_bytes(int32_t prec) { return prec == OIM_PREC_FP32 ? 8 : 4; }

constexpr size_t kSmemBudget = 227 * 1024 - 1024;

// Cost of one block (relative units) holding k replicas of graph g for one step:
// per node-replica work (noise, trig, update) plus per edge-update work.
static double block_cost(const GraphDev& gd, int64_t nnz_g, int k, int32_t prec) {
    const double per_node = 60.0, per_edge = (prec == OIM_PREC_FP32) ? 3.0 : 2.6;
    return (double)k * ((double)gd.n * per_node + (double)nnz_g * per_edge);
}

// Plan a resident launch: the kernel variant, per-graph replicas per block and
// the block list.  Quad kernel when four replicas of the largest graph fit;
// otherwise the pair/single kernel.  Without a requested k, each graph gets the
// k (multiple of the unit) that makes every block cost about the same while
// the whole grid stays within one wave of the SMs, as far as shared memory allows.
cudaError_t plan_resident(const oim_problem_s& p, int32_t R_pad, int32_t prec, int32_t want_k,
                          int32_t want_threads, ResidentPlan* plan) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 148;
    }
    const size_t cb = resident_cache_bytes(prec);
    const int G = p.G;
    std::vector<int64_t> nnz_g(G);
    for (int g = 0; g < G; ++g) {
        const int64_t end = (g + 1 < G) ? p.graphs[g + 1].edge_off : p.nnz;
        nnz_g[g] = end - p.graphs[g].edge_off;
    }
    // can the structure go to shared memory?  (+-1 weights, 15-bit local indices)
    bool csr_ok = p.unit_weights;
    std::vector<size_t> csr_bytes(G, 0);
    for (int g = 0; g < G; ++g) {
        if (p.graphs[g].n > 32767) csr_ok = false;
        csr_bytes[g] = align16((size_t)(p.graphs[g].n + 1) * 4) + align16((size_t)p.graphs[g].n * 4) +
                       align16((size_t)p.graphs[g].n * 2) + align16((size_t)nnz_g[g] * 2);
    }
    auto k_fit = [&](int g, bool with_csr) -> int {
        const size_t avail = kSmemBudget - (with_csr ? csr_bytes[g] : 0);
        if (avail > kSmemBudget) return 0;
        return (int)std::min<size_t>(64, avail / (cb * (size_t)p.graphs[g].n));
    };
    // unit: 4 (quad kernel) when every graph fits a quad, else 2 or 1
    int unit = 4;
    bool use_csr = csr_ok;
    for (int g = 0; g < G; ++g) {
        if (use_csr && k_fit(g, true) < 4) use_csr = false;
    }
    for (int g = 0; g < G; ++g) {
        const int f = k_fit(g, use_csr);
        if (f < unit) unit = f >= 2 ? 2 : (f >= 1 ? 1 : 0);
    }
    if (unit == 0) return cudaErrorInvalidValue;
    if (unit < 4) use_csr = false;
    std::vector<int> kg(G);
    for (int g = 0; g < G; ++g) kg[g] = (k_fit(g, use_csr) / unit) * unit;
    if (want_k > 0) {
        if (want_k % unit != 0) return cudaErrorInvalidValue;
        for (int g = 0; g < G; ++g) {
            if (want_k > kg[g]) return cudaErrorInvalidValue;
            kg[g] = want_k;
        }
    } else {
        // balance: smallest per-block cost tau such that the blocks fit in one wave
        auto blocks_for = [&](double tau, std::vector<int>& ks) {
            int64_t total = 0;
            for (int g = 0; g < G; ++g) {
                int k = unit;
                while (k + unit <= kg[g] && block_cost(p.graphs[g], nnz_g[g], k + unit, prec) <= tau)
                    k += unit;
                ks[g] = std::min(k, std::max(unit, R_pad));
                total += (R_pad + ks[g] - 1) / ks[g];
            }
            return total;
        };
        std::vector<int> ks(G);
        double lo = 0.0, hi = 0.0;
        for (int g = 0; g < G; ++g) hi = std::max(hi, block_cost(p.graphs[g], nnz_g[g], kg[g], prec));
        if (blocks_for(hi, ks) > sms) {
            blocks_for(hi, kg);   // more than one wave even at the largest k
        } else {
            for (int it = 0; it < 60; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (blocks_for(mid, ks) <= sms) hi = mid; else lo = mid;
            }
            blocks_for(hi, kg);
        }
    }
    plan->unit = unit;
    plan->csr_smem = use_csr;
    plan->k_of_graph = kg;
    plan->items.clear();
    size_t smem = 0;
    int max_units = 1;
    std::vector<std::pair<double, int4>> order;
    for (int g = 0; g < G; ++g) {
        const int k = std::min(kg[g], R_pad);
        for (int r0 = 0; r0 < R_pad; r0 += k) {
            const int kk = std::min(k, R_pad - r0);
            order.push_back({block_cost(p.graphs[g], nnz_g[g], kk, prec), make_int4(g, r0, kk, 0)});
        }
        smem = std::max(smem, (unit == 4 ? align16(cb * (size_t)p.graphs[g].n * k) : cb * (size_t)p.graphs[g].n * k) +
                                  (use_csr ? csr_bytes[g] : 0));
        max_units = std::max(max_units, k / unit);
    }
    // longest blocks first, so that a second wave (if any) fills in behind them
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) {
                         return x.first > y.first;
                     });
    for (auto& o : order) plan->items.push_back(o.second);
    int threads = want_threads > 0 ? want_threads : 1024;
    threads = std::min(1024, std::max(threads, 32 * ((max_units + 31) / 32)));
    if (want_threads <= 0) {
        const int64_t work = (int64_t)p.max_n * max_units;
        if (work < threads) threads = std::max(32, (int)((work + 31) / 32) * 32);
    }
    plan->threads = threads;
    plan->smem = smem;
    // the quad kernel's second (cos, sin) cache, where it fits beside everything else
    plan->double_buffer = false;
    if (unit == 4) {
        size_t smem_db = 0;
        for (int g = 0; g < G; ++g) {
            const int k = std::min(kg[g], R_pad);
            smem_db = std::max(smem_db, 2 * align16(cb * (size_t)p.graphs[g].n * k) + (use_csr ? csr_bytes[g] : 0));
        }
        if (smem_db <= kSmemBudget) {
            plan->double_buffer = true;
            plan->smem = smem_db;
        }
    }
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
    a.T = r.steps;
    a.double_buffer = r.plan.double_buffer ? 1 : 0;
    a.integer_weights = r.p->integer_weights ? 1 : 0;
    const ResidentPlan& pl = r.plan;
    const int blocks = (int)pl.items.size();
    const bool unit = r.p->unit_weights;
    if (pl.unit == 4) {
        if (r.prec == OIM_PREC_FP32)
            return launch_quad_v<QuadF32>(pl.csr_smem, unit, a, blocks, pl.threads, pl.smem, s);
        if (r.prec == OIM_PREC_FP16)
            return launch_quad_v<QuadF16>(pl.csr_smem, unit, a, blocks, pl.threads, pl.smem, s);
        return launch_quad_v<QuadBF16>(pl.csr_smem, unit, a, blocks, pl.threads, pl.smem, s);
    }
    if (r.prec == OIM_PREC_FP32)
        return launch_u<CacheF32>(pl.unit, unit, a, blocks, pl.threads, pl.smem, s);
    if (r.prec == OIM_PREC_FP16)
        return launch_u<CacheF16>(pl.unit, unit, a, blocks, pl.threads, pl.smem, s);
    return launch_u<CacheBF16>(pl.unit, unit, a, blocks, pl.threads, pl.smem, s);
}

}  // namespace oim

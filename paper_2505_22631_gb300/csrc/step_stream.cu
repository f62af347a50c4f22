// step_stream.cu -- the CSR stream form: one launch per Euler-Maruyama step, all
// state in device memory.  The plain form keeps the (cos, sin) cache in FP32 and
// uses correctly rounded math; the 16-bit variant stores the cache as FP16 or BF16
// pairs (half the cache bytes per step), recomputes each node's own (cos, sin) in
// FP32 from its phase, and uses the hardware approximations for the trigonometry
// and Box-Muller (errors ~1e-6, far below the 16-bit storage's 2^-11 / 2^-8).
//
// Layout: theta[node][R_pad] (FP32) and cs[node][R_pad] = (cos 2 pi theta,
// sin 2 pi theta), replicas contiguous.  In the plain form one thread owns one node
// and a quad of four consecutive replicas (two 16-byte loads per neighbour: a warp
// turns them into fully used 128-byte lines) and one Philox block feeds the quad's
// four noise draws.  In the 16-bit form one thread owns a node and an octet of eight
// consecutive replicas: one 32-byte load per neighbour, the row's index work shared
// by eight replicas, two Philox blocks sharing one key schedule.
//
// Per step and node (Eq. 5 / Algorithm 1, synchronous update from the old phases;
// the (cos, sin) cache the neighbours read is double-buffered as in Sec. III-B, and
// the phases are updated in place because a thread reads and writes only its own):
//   (A, B)   = sum_j w_ij (cos 2 pi theta_j, sin 2 pi theta_j)
//   D_i      = sin(2 pi theta_i) A - cos(2 pi theta_i) B = sum_j w_ij sin 2 pi (theta_i - theta_j)
//   theta_i' = wrap(theta_i + dt (K D_i - Ks sin 2 pi q theta_i) + Kn sqrt(dt) xi)
//   cs_i'    = (cos 2 pi theta_i', sin 2 pi theta_i')
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "oim_checks.cuh"
#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {

namespace {

// Storage of the (cos, sin) cache: four replicas' pairs per thread.
struct CacheF32 {
    using T = float2;
    static constexpr bool kOwnFromCache = true;   // the plain form reads its own pairs back
    static constexpr bool kFastMath = false;      // correctly rounded sincospi, logf, sqrtf
    static constexpr int kHead = 2;               // row-head entries taken from the descriptor
    __device__ static void load4(const T* p, float2 (&v)[4]) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
        v[2] = make_float2(b.x, b.y);
        v[3] = make_float2(b.z, b.w);
    }
    __device__ static void store4(T* p, const float2 (&v)[4]) {
        reinterpret_cast<float4*>(p)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        reinterpret_cast<float4*>(p)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    }
};

template <typename H2>
struct Cache16 {
    using T = H2;
    static constexpr bool kOwnFromCache = false;  // own pairs recomputed in FP32
    // hardware sin / cos / log2 / sqrt (errors ~1e-6, far below the 16-bit storage's)
    static constexpr bool kFastMath = true;
    __device__ static float2 to_f2(H2 h);
    __device__ static H2 from_f2(float2 f);
    __device__ static void store4(T* p, const float2 (&v)[4]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const H2 h = from_f2(v[k]);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
};

template <>
__device__ float2 Cache16<__half2>::to_f2(__half2 h) { return __half22float2(h); }
template <>
__device__ __half2 Cache16<__half2>::from_f2(float2 f) { return __floats2half2_rn(f.x, f.y); }
template <>
__device__ float2 Cache16<__nv_bfloat162>::to_f2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
template <>
__device__ __nv_bfloat162 Cache16<__nv_bfloat162>::from_f2(float2 f) { return __floats2bfloat162_rn(f.x, f.y); }

// Thread = node x quad of replicas: initial phases and their (cos, sin).
template <typename C>
__global__ void __launch_bounds__(128) init_stream_kernel(CSRDev csr, StepParams P,
                                                          float* __restrict__ theta,
                                                          typename C::T* __restrict__ cs) {
    const int quads = P.R_pad >> 2;
    const int node = blockIdx.x * blockDim.y + threadIdx.y;
    const int quad = blockIdx.y * blockDim.x + threadIdx.x;
    if (node >= csr.nodes || quad >= quads) return;
    const int r = 4 * quad;
    const int g = csr.node_graph[node];
    const int i = node - csr.graphs[g].node_off;
    const uint64_t seed = P.seed_dev ? *P.seed_dev : P.seed;
    const float2 t01 = init_pair(seed, (uint32_t)g, (uint32_t)i, (uint32_t)r);
    const float2 t23 = init_pair(seed, (uint32_t)g, (uint32_t)i, (uint32_t)(r + 2));
    const size_t at = (size_t)node * P.R_pad + r;
    *reinterpret_cast<float4*>(theta + at) = make_float4(t01.x, t01.y, t23.x, t23.y);
    const float th[4] = {t01.x, t01.y, t23.x, t23.y};
    float2 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (C::kFastMath)   // the 16-bit caches hold half-turn pairs (see step_octet_kernel)
            v[k] = cos_sin_half_turn_fast(th[k]);
        else
            sincospif(2.0f * th[k], &v[k].y, &v[k].x);
    }
    C::store4(cs + at, v);
}

// The plain form (FP32 cache): thread = node x quad of replicas.  kAB: the coupling
// sums (A, B) of the step are also stored at ab[node][R_pad] (the schedule adjoint's
// recomputation keeps them, so its reverse sweep gathers only the lambda-weighted pairs).
template <bool kUnit, typename C, bool kAB = false>
__global__ void __launch_bounds__(128) step_stream_kernel(CSRDev csr, StepParams P, const float* th_in,
                                                          const typename C::T* __restrict__ cs_in,
                                                          float* th_out,
                                                          typename C::T* __restrict__ cs_out,
                                                          int64_t t_fixed,
                                                          const int32_t* __restrict__ d_t0,
                                                          int32_t t_add, int quads_fast,
                                                          float2* __restrict__ ab = nullptr) {
    // block = blockDim.x replica quads x blockDim.y nodes (no index division); the
    // blocks take their nodes in the batch's heaviest-rows-first order, and with
    // quads_fast the grid's fast dimension runs over replica blocks, so the blocks
    // are dispatched longest first and the short rows fill the tail
    const int quads = P.R_pad >> 2;
    const int nblk = quads_fast ? blockIdx.y : blockIdx.x;
    const int qblk = quads_fast ? blockIdx.x : blockIdx.y;
    const int slot = nblk * blockDim.y + threadIdx.y;
    const int quad = qblk * blockDim.x + threadIdx.x;
    if (slot >= csr.nodes || quad >= quads) return;
    const int4 row = __ldg(csr.srow + slot);   // {node, row start, first -1 entry, row end}
    const int node = row.x;

    float2 acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] = make_float2(0.f, 0.f);
    const int e_beg = row.y, e_end = row.w;
    constexpr int kH = C::kHead;
    {
        // the head entries' pairs: their column words come with the slot's descriptor
        const uint4 hd = __ldg(csr.shead + slot);
        const uint32_t hc[4] = {hd.x, hd.y, hd.z, hd.w};
        float2 hv[kH][4];
#pragma unroll
        for (int u = 0; u < kH; ++u)
            C::load4(cs_in + (size_t)checked_node_of_row(csr, node, kUnit ? (hc[u] & ~kSignBit) : hc[u]) * P.R_pad +
                         4 * quad,
                     hv[u]);
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            if (e_beg + u < e_end) {
                const float w = kUnit ? ((hc[u] & kSignBit) ? -1.0f : 1.0f) : __ldg(csr.w + e_beg + u);
                const float2 ww = make_float2(w, w);
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[v] = ffma2(hv[u][v], ww, acc[v]);
            }
        }
    }
    for (int e = e_beg + kH; e < e_end; ++e) {
        const uint32_t cw = __ldg(csr.col + e);
        float w;
        uint32_t j;
        if (kUnit) {
            j = cw & ~kSignBit;
            w = (cw & kSignBit) ? -1.0f : 1.0f;
        } else {
            j = cw;
            w = __ldg(csr.w + e);
        }
        j = checked_node_of_row(csr, node, j);
        float2 nb[4];
        C::load4(cs_in + (size_t)j * P.R_pad + 4 * quad, nb);
        const float2 ww = make_float2(w, w);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] = ffma2(nb[v], ww, acc[v]);
    }

    // the node's own state after the gather: only the gather's state is live during it
    const int g = csr.node_graph[node];
    const int i = node - csr.graphs[g].node_off;
    const int64_t t = d_t0 ? (int64_t)(*d_t0) + t_add : t_fixed;
    const size_t sidx = (size_t)g * P.steps + t;
    const float K = __ldg(P.K + sidx), Ks = __ldg(P.Ks + sidx), Kn = __ldg(P.Kn + sidx);
    const size_t at = (size_t)node * P.R_pad + 4 * quad;
    const float4 th = *reinterpret_cast<const float4*>(th_in + at);
    const float t0[4] = {th.x, th.y, th.z, th.w};
    float2 own[4];
    C::load4(cs_in + at, own);
    const uint4 x = draw_block(P.seed_dev ? *P.seed_dev : P.seed, (uint32_t)g, kStreamNoise, (uint32_t)i,
                               (uint32_t)t, (uint32_t)quad);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float z[4] = {z01.x, z01.y, z23.x, z23.y};
    const float kick = Kn * P.sqrt_dt;
    const float dtK = P.dt * K, dtKs = P.dt * Ks;
    float tn[4];
    float2 ncs[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float coup = own[v].y * acc[v].x - own[v].x * acc[v].y;
        const float shil = sin_q(P.q, own[v].x, own[v].y);
        tn[v] = wrap01(t0[v] + (dtK * coup - dtKs * shil) + kick * z[v]);
        sincospif(2.0f * tn[v], &ncs[v].y, &ncs[v].x);
    }
    *reinterpret_cast<float4*>(th_out + at) = make_float4(tn[0], tn[1], tn[2], tn[3]);
    C::store4(cs_out + at, ncs);
    if constexpr (kAB) {
        reinterpret_cast<float4*>(ab + at)[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
        reinterpret_cast<float4*>(ab + at)[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
    }
}

// Eight 16-bit (cos, sin) pairs added to, or subtracted from, the accumulators.
template <typename H2>
__device__ __forceinline__ void add8(float2 (&acc)[8], const uint32_t (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if constexpr (std::is_same<H2, __half2>::value) add_f16x2(acc[k], v[k]);
        else add_bf16x2(acc[k], v[k]);
    }
}
template <typename H2>
__device__ __forceinline__ void rsub8(float2 (&acc)[8], const uint32_t (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if constexpr (std::is_same<H2, __half2>::value) rsub_f16x2(acc[k], v[k]);
        else rsub_bf16x2(acc[k], v[k]);
    }
}
template <typename H2>
__device__ __forceinline__ float2 h2_to_f2(uint32_t h) {
    if constexpr (std::is_same<H2, __half2>::value) return __half22float2(*reinterpret_cast<const __half2*>(&h));
    else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h));
}
template <typename H2>
__device__ __forceinline__ uint32_t f2_to_h2(float2 f) {
    if constexpr (std::is_same<H2, __half2>::value) {
        const __half2 h = __floats2half2_rn(f.x, f.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f.x, f.y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

constexpr int kOctetThreads = 128;   // threads per block of the per-step 16-bit kernel

// The 16-bit form: thread = node x octet of eight consecutive replicas.  A slot's
// 32-byte descriptor {node, row start, first -1 entry, row end, graph, local index,
// first two column indices} arrives in one load, so the first two neighbours' pairs
// are requested one dependent load after launch and the node's graph and Philox
// counter need no further lookups.
//
// The 16-bit cache holds half-turn pairs (cos, sin)(2 pi (theta + 1/2)) =
// -(cos, sin)(2 pi theta), whose argument reduction is one FMA; with the node's own
// pair taken the same way the coupling s A - c B is unchanged, the injection
// sin 2 pi q (theta + 1/2) = (-1)^q sin 2 pi q theta and the Box-Muller normals of the
// shifted angle are negated, both folded into their scalar factors (exact).
//
// +-1 weights (kUnit): the row holds its +1 entries first.  They are added with mixed
// f16 + f32 adds (one rounding each, as the FMA by +1 would give); the first -1 entry
// is taken with the mixed subtract acc = x - acc, which negates the accumulator, and
// the rest of the -1 run is added to the negated accumulator:
// -(acc - x1 - x2) = (x1 - acc) + x2, each rounding to nearest exactly as the FMAs by -1
// would.  The sign is folded into dt K at the end (exact).  Other weights: each pair
// is converted to FP32 and multiply-added.
// 48 registers: 40 warps an SM to cover the gather's latency (measured on the two-graph
// benchmark batch: 64 registers 19.9 us, 48 registers 18.6 us per step; 40 registers
// spill), in blocks of 128 threads (ten an SM): a block's slot frees as soon as its four
// nodes are done, which leaves fewer warp slots idle behind a block's slowest warp than
// blocks of eight nodes (16.95 against 17.28 us per step on the benchmark batch, 124.4
// against 127.8 on the 16-graph batch; 64 threads: 17.00 / 123.2)
// One step of one (slot, octet) work item.  kCoherent: the neighbours' pairs are read
// through L2 only (ld.global.cg), for the persistent kernel, whose pairs were written
// by other blocks during the same launch; the per-step kernel reads them through the
// read-only path.
// A 32-byte load through L2 only (not kept in L1).
__device__ __forceinline__ void ld256_l2(const void* p, uint32_t (&r)[8]) {
    asm("ld.global.cg.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}

template <typename H2, bool kUnit, int kQ, bool kCoherent, bool kPre = false>
__device__ __forceinline__ void octet_step(const CSRDev& csr, const StepParams& P, float* theta,
                                           const H2* __restrict__ cs_in, H2* __restrict__ cs_out,
                                           int slot, int oct, int64_t t_fixed,
                                           const int32_t* __restrict__ d_t0, int32_t t_add,
                                           uint4 xa_pre = uint4{}, uint4 xb_pre = uint4{}) {
    auto ld_pairs = [](const char* p, uint32_t (&r)[8]) {
        if constexpr (kCoherent) ld256_cg(p, r);
        else ld256_nc(p, r);
    };
    uint32_t d[8];
    ld256_nc(csr.sdesc + (size_t)slot * 8, d);
    const int node = (int)d[0], e_beg = (int)d[1], e_split = (int)d[2], e_end = (int)d[3];
    // (checked builds: every column a node of the row's graph d[4])
    auto col = [&](uint32_t j) { return checked_node(csr, (int)d[4], j, (uint32_t)node); };
    const char* cs_base = reinterpret_cast<const char*>(cs_in) + (size_t)oct * 32;
    // bytes per node row (R_pad <= 2^20: 32 bits), so that a neighbour's address is one
    // 32 x 32 -> 64-bit multiply-add
    const uint32_t stride = (uint32_t)P.R_pad * (uint32_t)sizeof(uint32_t);
    float2 acc[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] = make_float2(0.f, 0.f);
    float sgn = 1.0f;
    if constexpr (kUnit) {
        uint32_t h0[8], h1[8];
        ld_pairs(cs_base + (size_t)col(d[6]) * stride, h0);
        ld_pairs(cs_base + (size_t)col(d[7]) * stride, h1);
        if (e_beg < e_end) {
            if (e_beg == e_split) rsub8<H2>(acc, h0);
            else add8<H2>(acc, h0);
        }
        if (e_beg + 1 < e_end) {
            if (e_beg + 1 == e_split) rsub8<H2>(acc, h1);
            else add8<H2>(acc, h1);
        }
        int e = e_beg + 2;
        const uint32_t* cp = reinterpret_cast<const uint32_t*>(csr.pcol) + e;
        for (; e < e_split; ++e, ++cp) {
            uint32_t v[8];
            ld_pairs(cs_base + (size_t)col(__ldg(cp)) * stride, v);
            add8<H2>(acc, v);
        }
        if (e == e_split && e < e_end) {
            uint32_t v[8];
            ld_pairs(cs_base + (size_t)col(__ldg(cp)) * stride, v);
            rsub8<H2>(acc, v);
            ++e;
            ++cp;
        }
        for (; e < e_end; ++e, ++cp) {
            uint32_t v[8];
            ld_pairs(cs_base + (size_t)col(__ldg(cp)) * stride, v);
            add8<H2>(acc, v);
        }
        if (e_split < e_end) sgn = -1.0f;   // the accumulators hold -(A, B)
    } else {
        for (int e = e_beg; e < e_end; ++e) {
            uint32_t v[8];
            ld_pairs(cs_base + (size_t)col((uint32_t)__ldg(csr.pcol + e)) * stride, v);
            const float w = __ldg(csr.w + e);
            const float2 ww = make_float2(w, w);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = ffma2(h2_to_f2<H2>(v[k]), ww, acc[k]);
        }
    }

    const int g = (int)d[4], i = (int)d[5];
    const int64_t t = d_t0 ? (int64_t)(*d_t0) + t_add : t_fixed;
    const size_t sidx = (size_t)g * P.steps + t;
    const float K = __ldg(P.K + sidx), Ks = __ldg(P.Ks + sidx), Kn = __ldg(P.Kn + sidx);
    const size_t at = (size_t)node * P.R_pad + 8 * oct;
    // own phases through L2 (they are read once): another block's store of the previous
    // step to the same 128-byte line (fewer than 32 replicas a node) can then never be
    // met in a stale L1 copy, also when this step's blocks start while the previous
    // step still runs (programmatic dependent launch)
    uint32_t thw[8];
    if constexpr (kCoherent) ld256_cg(theta + at, thw);   // ordered against the previous step's store
    else ld256_l2(theta + at, thw);
    uint4 xa = xa_pre, xb = xb_pre;   // kPre: drawn by the caller
    if constexpr (!kPre) {
        const uint64_t seed = P.seed_dev ? *P.seed_dev : P.seed;
        draw_block_pair(seed, (uint32_t)g, kStreamNoise, (uint32_t)i, (uint32_t)t, (uint32_t)(2 * oct), xa, xb);
    }
    float z[8];   // the negated normals
    {
        const float2 z0 = box_muller_half_turn_fast(xa.x, xa.y), z1 = box_muller_half_turn_fast(xa.z, xa.w);
        const float2 z2 = box_muller_half_turn_fast(xb.x, xb.y), z3 = box_muller_half_turn_fast(xb.z, xb.w);
        z[0] = z0.x; z[1] = z0.y; z[2] = z1.x; z[3] = z1.y;
        z[4] = z2.x; z[5] = z2.y; z[6] = z3.x; z[7] = z3.y;
    }
    const int q = kQ > 0 ? kQ : P.q;
    const float kick = -(Kn * P.sqrt_dt);
    const float dtK = (P.dt * K) * sgn;
    // q = 2: sin 4 pi theta = 2 s c, the 2 taken into the factor (exact)
    const float dtKs = (kQ == 2 ? 2.0f : 1.0f) * ((q & 1) ? -(P.dt * Ks) : P.dt * Ks);
    // replica pairs in packed FP32 (the same roundings, in the same order, as the
    // scalar expression th + (dtK coup - dtKs shil) + kick z)
    uint32_t tno[8], cso[8];
    const float2 dtK2 = make_float2(dtK, dtK), ndtKs2 = make_float2(-dtKs, -dtKs), kick2 = make_float2(kick, kick);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float th0 = __uint_as_float(thw[2 * p]), th1 = __uint_as_float(thw[2 * p + 1]);
        const float2 o0 = cos_sin_half_turn_fast(th0), o1 = cos_sin_half_turn_fast(th1);
        const float2 S = make_float2(o0.y, o1.y), C = make_float2(o0.x, o1.x);
        const float2 A = make_float2(acc[2 * p].x, acc[2 * p + 1].x), B = make_float2(acc[2 * p].y, acc[2 * p + 1].y);
        const float2 coup = __ffma2_rn(S, A, __fmul2_rn(make_float2(-C.x, -C.y), B));
        const float2 shil = kQ == 2 ? __fmul2_rn(C, S) : make_float2(sin_q(q, o0.x, o0.y), sin_q(q, o1.x, o1.y));
        const float2 inc = __ffma2_rn(dtK2, coup, __fmul2_rn(ndtKs2, shil));
        const float2 x = __ffma2_rn(kick2, make_float2(z[2 * p], z[2 * p + 1]), __fadd2_rn(make_float2(th0, th1), inc));
        const float tn0 = wrap01(x.x), tn1 = wrap01(x.y);
        tno[2 * p] = __float_as_uint(tn0);
        tno[2 * p + 1] = __float_as_uint(tn1);
        cso[2 * p] = f2_to_h2<H2>(cos_sin_half_turn_fast(tn0));
        cso[2 * p + 1] = f2_to_h2<H2>(cos_sin_half_turn_fast(tn1));
    }
    st256(theta + at, tno);
    st256(cs_out + at, cso);
}

// After griddepcontrol.wait: the state pointers pass through a volatile move, so that
// no load through them (the 256-bit loads are plain asm, which the compiler may move
// across other asm) can be scheduled before the wait.
template <typename T>
__device__ __forceinline__ T* after_wait(T* p) {
    uint64_t v = reinterpret_cast<uint64_t>(p);
    asm volatile("mov.b64 %0, %0;" : "+l"(v));
    return reinterpret_cast<T*>(v);
}

template <typename H2, bool kUnit, int kQ>
__global__ void __launch_bounds__(kOctetThreads, 10) step_octet_kernel(CSRDev csr, StepParams P, float* theta,
                                                            const H2* __restrict__ cs_in,
                                                            H2* __restrict__ cs_out, int64_t t_fixed,
                                                            const int32_t* __restrict__ d_t0,
                                                            int32_t t_add, int octs_fast) {
    // launched as a programmatic dependent of the previous kernel in the stream: every
    // block waits (griddepcontrol.wait) for the previous grid's completion (and its
    // memory) before it reads anything a kernel writes (a no-op under a plain launch),
    // and only then lets the next step be scheduled (griddepcontrol.launch_dependents),
    // so that no step is launched before the step two back has finished reading the
    // (cos, sin) buffer the next one will read
    const int octs = P.R_pad >> 3;
    const int nblk = octs_fast ? blockIdx.y : blockIdx.x;
    const int oblk = octs_fast ? blockIdx.x : blockIdx.y;
    const int slot = nblk * blockDim.y + threadIdx.y;
    const int oct = oblk * blockDim.x + threadIdx.x;
    if (slot >= csr.nodes || oct >= octs) return;
    if (d_t0 == nullptr) {
        // the step is known: the noise depends on no kernel's output (the descriptors,
        // the seed and the schedules are written before the run), so it is drawn while
        // the previous step may still be running
        const uint32_t* dsc = csr.sdesc + (size_t)slot * 8;
        const uint64_t seed = P.seed_dev ? *P.seed_dev : P.seed;
        uint4 xa, xb;
        draw_block_pair(seed, __ldg(dsc + 4), kStreamNoise, __ldg(dsc + 5), (uint32_t)t_fixed, (uint32_t)(2 * oct),
                        xa, xb);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        octet_step<H2, kUnit, kQ, false, true>(csr, P, after_wait(theta), after_wait(cs_in), cs_out, slot, oct,
                                               t_fixed, d_t0, t_add, xa, xb);
    } else {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        octet_step<H2, kUnit, kQ, false>(csr, P, after_wait(theta), after_wait(cs_in), cs_out, slot, oct, t_fixed,
                                         after_wait(d_t0), t_add);
    }
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int32_t kErrGridBarrier = 16;           // error word: a grid barrier gave up
constexpr uint64_t kGridBarrierNs = 2000000000ull;  // two seconds

// Barrier of all blocks of a cooperative launch (co-resident by construction).  The last
// block to arrive resets the count and moves the generation on; the others wait for the
// generation to change for at most kGridBarrierNs, after which they record the error and
// the kernel returns.  The fences order every write of the block before its arrival and
// every later read after the wait (the bar.sync around them carries the block's threads).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int32_t* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned* vgen = gen;
        const unsigned g0 = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
            ok = 1;
        } else {
            ok = 1;
            const uint64_t start = global_ns();
            while (*vgen == g0) {
                if (global_ns() - start > kGridBarrierNs || *reinterpret_cast<volatile int32_t*>(err) != 0) {
                    atomicCAS(err, 0, kErrGridBarrier);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// The persistent form: steps [t0, t1) of the 16-bit stream form in one cooperative
// launch.  Each block walks the per-step kernel's blocks (same shape, same heaviest-first
// order) with a stride of the grid, then all blocks meet at a grid barrier before the
// next step reads the pairs this one wrote.
template <typename H2, bool kUnit, int kQ>
__global__ void __launch_bounds__(256, 5) step_octet_persistent_kernel(
    CSRDev csr, StepParams P, float* theta, H2* cs0, H2* cs1, int64_t t0, int64_t t1, int gx, int gy,
    unsigned* bar, int32_t* err) {
    const int octs = P.R_pad >> 3;
    const int vblocks = gx * gy;
    for (int64_t t = t0; t < t1; ++t) {
        const H2* cs_in = (t & 1) ? cs1 : cs0;
        H2* cs_out = (t & 1) ? cs0 : cs1;
        for (int vb = blockIdx.x; vb < vblocks; vb += gridDim.x) {
            const int oblk = vb % gx, nblk = vb / gx;   // replica blocks fastest, as octs_fast
            const int slot = nblk * blockDim.y + threadIdx.y;
            const int oct = oblk * blockDim.x + threadIdx.x;
            if (slot < csr.nodes && oct < octs)
                octet_step<H2, kUnit, kQ, true>(csr, P, theta, cs_in, cs_out, slot, oct, t, nullptr, 0);
        }
        if (t + 1 < t1 && !grid_barrier(bar, bar + 1, gridDim.x, err)) return;
    }
}

// f = K sum_j w_ij (s_i c_j - c_i s_j) - Ks sin(2 pi q theta_i) for theta[r][n] of
// one graph, with the same trig-cache identity and FP32 arithmetic as the steps.
__global__ void derivative_kernel(CSRDev csr, int q, int R, const float* __restrict__ theta,
                                  float K, float Ks, float* __restrict__ f) {
    const int n = csr.nodes;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * R) return;
    const int r = (int)(gid / n), i = (int)(gid - (int64_t)r * n);
    float si, ci;
    sincospif(2.0f * theta[gid], &si, &ci);
    float2 acc = make_float2(0.f, 0.f);
    for (int e = csr.rowp[i]; e < csr.rowp[i + 1]; ++e) {
        const uint32_t cw = csr.col[e];
        const uint32_t j = checked_local(csr, n, (int)(csr.w ? cw : (cw & ~kSignBit)), i);
        const float w = csr.w ? csr.w[e] : ((cw & kSignBit) ? -1.0f : 1.0f);
        float sj, cj;
        sincospif(2.0f * theta[(int64_t)r * n + j], &sj, &cj);
        acc = ffma2(make_float2(cj, sj), make_float2(w, w), acc);
    }
    f[gid] = K * (si * acc.x - ci * acc.y) - Ks * sin_q(q, ci, si);
}

}  // namespace

cudaError_t launch_derivative(const oim_problem_s& p, const float* theta, int32_t R, float K,
                              float Ks, float* f, cudaStream_t s) {
    const int64_t total = p.nodes * R;
    derivative_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p.csr(), p.q, R, theta, K,
                                                                       Ks, f);
    return cudaGetLastError();
}

// The run's seed into device memory, ordered on the stream before the run's kernels
// (a kernel argument is taken by value at launch, so the host needs no staging copy).
__global__ void set_seed_kernel(uint64_t* d_seed, uint64_t seed) { *d_seed = seed; }

cudaError_t launch_set_seed(uint64_t* d_seed, uint64_t seed, cudaStream_t s) {
    set_seed_kernel<<<1, 1, 0, s>>>(d_seed, seed);
    return cudaGetLastError();
}

// Launch shape of the thread = (node, replica quad) kernels: blocks of 128 threads (the
// persistent kernel: 256, which its grid barrier prefers), x over quads (a warp covers
// consecutive quads of a node: coalesced rows), y over nodes; the grid runs nodes along x
// (up to 2^31 - 1 blocks) and quads along y.  Blocks of 128 free their slot sooner than
// blocks of 256 (plain FP32 step on the benchmark batch 35.9 -> 35.3 us).
struct QuadGrid {
    dim3 grid, block;
};
static QuadGrid quad_grid(int64_t nodes, int quads, int threads = 128) {
    int qx = 1;
    while (qx < quads && qx < 32) qx <<= 1;
    const int ny = threads / qx;
    QuadGrid q;
    q.block = dim3((unsigned)qx, (unsigned)ny);
    q.grid = dim3((unsigned)((nodes + ny - 1) / ny), (unsigned)((quads + qx - 1) / qx));
    return q;
}

// The step kernels' grid: node blocks along x (dispatched first, heaviest rows first) and
// replica blocks along y, quads_fast = 0: the blocks that run at the same time then work
// on one replica range.  17.03 -> 16.77 us per step for the 16-bit kernel and 35.4 -> 34.3
// for the FP32 one on the benchmark batch, against replica blocks along x (quads_fast = 1),
// which put every replica block of the heaviest rows first (ncu on the 16-bit kernel:
// long-scoreboard stalls 9.05 -> 8.57 cycles per issue, L2 hit rate 66.5 -> 67.7 %).  The
// kernels keep both orientations (quads_fast a launch argument).
struct StepGrid {
    dim3 grid, block;
    int quads_fast;
};
static StepGrid step_grid(int64_t nodes, int quads, int threads = 128) {
    const QuadGrid q = quad_grid(nodes, quads, threads);
    return StepGrid{q.grid, q.block, 0};
}

static StepParams params_of(const oim_run_s& r) {
    StepParams P;
    const int G = r.p->G;
    P.K = r.d_sched;
    P.Ks = r.d_sched + (size_t)G * r.steps_cap;
    P.Kn = r.d_sched + (size_t)2 * G * r.steps_cap;
    P.steps = r.steps_cap;
    P.dt = r.dt;
    P.sqrt_dt = sqrtf(r.dt);
    P.seed = r.seed;
    P.seed_dev = r.d_seed;
    P.q = r.p->q;
    P.R = r.R;
    P.R_pad = r.R_pad;
    return P;
}

StepParams make_params(const oim_run_s& r) { return params_of(r); }

template <typename C>
static cudaError_t init_stream_as(const oim_run_s& r, cudaStream_t s) {
    const StepParams P = params_of(r);
    const QuadGrid q = quad_grid(r.p->nodes, r.R_pad / 4);
    init_stream_kernel<C><<<q.grid, q.block, 0, s>>>(
        r.p->csr(), P, r.d_theta[0], reinterpret_cast<typename C::T*>(r.d_cs[0]));
    return cudaGetLastError();
}

cudaError_t launch_init_stream(const oim_run_s& r, cudaStream_t s) {
    if (r.prec == OIM_PREC_FP16) return init_stream_as<Cache16<__half2>>(r, s);
    if (r.prec == OIM_PREC_BF16) return init_stream_as<Cache16<__nv_bfloat162>>(r, s);
    return init_stream_as<CacheF32>(r, s);
}

// (cos, sin) of every phase, for restarting the stream form from stored phases.
__global__ void cs_from_theta_kernel(int64_t count, const float* __restrict__ theta,
                                     float2* __restrict__ cs) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= count) return;
    float s, c;
    sincospif(2.0f * theta[gid], &s, &c);
    cs[gid] = make_float2(c, s);
}

cudaError_t launch_cs_from_theta(const oim_run_s& r, const float* theta, float2* cs, cudaStream_t s) {
    const int64_t count = r.p->nodes * r.R_pad;
    cs_from_theta_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, theta, cs);
    return cudaGetLastError();
}

// One step t of the stream form between explicit buffers (FP32 cache: the adjoint).
cudaError_t launch_step_stream_buffers(const oim_run_s& r, int64_t t, const float* th_in,
                                       const float2* cs_in, float* th_out, float2* cs_out, float2* ab,
                                       cudaStream_t s) {
    const StepParams P = params_of(r);
    const StepGrid q = step_grid(r.p->nodes, r.R_pad / 4);
    if (r.p->unit_weights)
        step_stream_kernel<true, CacheF32, true><<<q.grid, q.block, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, nullptr, 0, q.quads_fast, ab);
    else
        step_stream_kernel<false, CacheF32, true><<<q.grid, q.block, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, nullptr, 0, q.quads_fast, ab);
    return cudaGetLastError();
}

// The plain form's step t (FP32 cache).
static cudaError_t step_plain(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    // with d_t0 the step is *d_t0 + t (graph replay); otherwise t itself.
    const StepParams P = params_of(r);
    const CSRDev csr = step_csr(r);
    const StepGrid q = step_grid(csr.nodes, r.R_pad / 4);
    const int in = (int)(t & 1);   // buffer parity follows the step index
    const int out = in ^ 1;
    const float* th_in = r.d_theta[in];
    const float2* cs_in = reinterpret_cast<const float2*>(r.d_cs[in]);
    float* th_out = r.d_theta[out];
    float2* cs_out = reinterpret_cast<float2*>(r.d_cs[out]);
    if (r.p->unit_weights)
        step_stream_kernel<true, CacheF32><<<q.grid, q.block, 0, s>>>(
            csr, P, th_in, cs_in, th_out, cs_out, t, d_t0, (int32_t)t, q.quads_fast);
    else
        step_stream_kernel<false, CacheF32><<<q.grid, q.block, 0, s>>>(
            csr, P, th_in, cs_in, th_out, cs_out, t, d_t0, (int32_t)t, q.quads_fast);
    return cudaGetLastError();
}

// The 16-bit form's step t: thread = node x octet of replicas (R_pad a multiple of 8).
// (launched with programmatic stream serialization: consecutive steps overlap the next
// launch with the tail of the previous one; in a captured graph the edge is programmatic)
template <typename H2, int kQ>
static cudaError_t step_octet_q(const oim_run_s& r, const CSRDev& csr, const StepParams& P, const StepGrid& q,
                                float* theta, const H2* cs_in, H2* cs_out, int64_t t, const int32_t* d_t0,
                                cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = q.grid;
    cfg.blockDim = q.block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int32_t t_add = (int32_t)t;
    const int octs_fast = q.quads_fast;
    if (r.p->unit_weights)
        return cudaLaunchKernelEx(&cfg, step_octet_kernel<H2, true, kQ>, csr, P, theta, cs_in, cs_out, t, d_t0,
                                  t_add, octs_fast);
    return cudaLaunchKernelEx(&cfg, step_octet_kernel<H2, false, kQ>, csr, P, theta, cs_in, cs_out, t, d_t0,
                              t_add, octs_fast);
}

template <typename H2>
static cudaError_t step_octet(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    const StepParams P = params_of(r);
    const CSRDev csr = step_csr(r);
    const StepGrid q = step_grid(csr.nodes, r.R_pad / 8, kOctetThreads);
    const int in = (int)(t & 1);
    // phases in place (one buffer), the (cos, sin) pairs double-buffered
    float* theta = r.d_theta[in];
    const H2* cs_in = reinterpret_cast<const H2*>(r.d_cs[in]);
    H2* cs_out = reinterpret_cast<H2*>(r.d_cs[in ^ 1]);
    if (P.q == 2) return step_octet_q<H2, 2>(r, csr, P, q, theta, cs_in, cs_out, t, d_t0, s);
    if (P.q == 3) return step_octet_q<H2, 3>(r, csr, P, q, theta, cs_in, cs_out, t, d_t0, s);
    return step_octet_q<H2, 0>(r, csr, P, q, theta, cs_in, cs_out, t, d_t0, s);
}

// Steps [t0, t1) of the 16-bit stream form in one cooperative launch of as many blocks
// as fit on the GPU at once (the per-step kernel's blocks are walked with their stride).
template <typename H2, bool kUnit, int kQ>
static cudaError_t persistent_as(const oim_run_s& r, int64_t t0, int64_t t1, cudaStream_t s) {
    const StepParams P = params_of(r);
    const CSRDev csr = step_csr(r);
    const StepGrid q = step_grid(csr.nodes, r.R_pad / 8, 256);
    int gx = (int)q.grid.x, gy = (int)q.grid.y;   // octet blocks, node blocks
    if (!q.quads_fast) std::swap(gx, gy);
    auto fn = step_octet_persistent_kernel<H2, kUnit, kQ>;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)(q.block.x * q.block.y), 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(per_sm * sms, gx * gy));
    H2* cs0 = reinterpret_cast<H2*>(r.d_cs[0]);
    H2* cs1 = reinterpret_cast<H2*>(r.d_cs[1]);
    float* theta = r.d_theta[0];
    unsigned* bar = r.d_bar;
    int32_t* err = r.d_err;
    void* args[] = {const_cast<CSRDev*>(&csr), const_cast<StepParams*>(&P), &theta, &cs0, &cs1, &t0, &t1,
                    &gx, &gy, &bar, &err};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3((unsigned)blocks), q.block, args,
                                       0, s);
}

template <typename H2>
static cudaError_t persistent_h2(const oim_run_s& r, int64_t t0, int64_t t1, cudaStream_t s) {
    const int q = r.p->q;
    if (r.p->unit_weights) {
        if (q == 2) return persistent_as<H2, true, 2>(r, t0, t1, s);
        if (q == 3) return persistent_as<H2, true, 3>(r, t0, t1, s);
        return persistent_as<H2, true, 0>(r, t0, t1, s);
    }
    if (q == 2) return persistent_as<H2, false, 2>(r, t0, t1, s);
    if (q == 3) return persistent_as<H2, false, 3>(r, t0, t1, s);
    return persistent_as<H2, false, 0>(r, t0, t1, s);
}

cudaError_t launch_persistent_steps(const oim_run_s& r, int64_t t0, int64_t t1, cudaStream_t s) {
    if (t1 <= t0) return cudaSuccess;
    if (r.prec == OIM_PREC_BF16) return persistent_h2<__nv_bfloat162>(r, t0, t1, s);
    return persistent_h2<__half2>(r, t0, t1, s);
}

cudaError_t launch_step_stream(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    if (r.prec == OIM_PREC_FP16) return step_octet<__half2>(r, t, d_t0, s);
    if (r.prec == OIM_PREC_BF16) return step_octet<__nv_bfloat162>(r, t, d_t0, s);
    return step_plain(r, t, d_t0, s);
}

}  // namespace oim

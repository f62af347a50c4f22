// gemm_step.cu -- the dense coupling form: one Euler-Maruyama step per launch with
// the coupling sums on the tensor cores.
//
// With X^T = [cos 2 pi theta ; sin 2 pi theta] (rows 2r and 2r + 1 for replica r,
// columns = nodes, BF16) and W the dense coupling matrix (BF16; +-1 weights are
// exact), one step needs D^T = X^T W, i.e. D^T[2r][i] = A_{i,r} = sum_j w_ij c_j,r and
// D^T[2r+1][i] = B_{i,r}; W is symmetric, so W itself is the K-major B operand.
// A CTA computes a 128 x 128 tile of D^T with tcgen05.mma (FP32 accumulator in
// TMEM) from TMA-loaded 128-byte-swizzled tiles, and its eight epilogue warps finish
// the step for the tile's (node, replica) pairs: coupling s A - c B, injection,
// Philox noise, Euler update and wrap (Eq. 5, Algorithm 1), writing the new FP32
// phases ([R_pad][n_pad], replica-major) and the next step's BF16 X^T.
// The trigonometry and Box-Muller use the hardware approximations (the BF16
// operands round at 2^-9, far above their ~1e-6 error).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "oim_checks.cuh"
#include "oim_device.cuh"
#include "oim_internal.h"
#include "tc_common.cuh"

namespace oim {

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int make_map_bf16(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t pitch,
                  uint32_t box_rows);

namespace {

constexpr int kBM = 128, kBK = 64, kABytes = kBM * 128;

struct GemmArgs {
    float* theta;               // [R_pad][n_pad], updated in place
    __nv_bfloat16* x_out;       // [2 R_pad][n_pad], next step's X^T
    const float* K;             // schedules of this graph, indexed by t
    const float* Ks;
    const float* Kn;
    int64_t t;                  // the step, or its offset from *t0 when t0 is set
    const int32_t* t0;          // step base in device memory (a replayed chunk of steps)
    float dt, sqrt_dt;
    const uint64_t* seed;       // device copy of the run's seed (graph replays serve any seed)
    int32_t graph, q, n, n_pad;
    int32_t* err;
};

// Block layout: warp 0 lane 0 streams the K blocks with TMA, warp 1 lane 0 issues the
// MMAs, the remaining warps are the epilogue.  TMEM lanes are split by warp index
// mod 4, so the epilogue warps cover the four 32-lane quadrants once per 64-column
// part of the tile: warp w takes quadrant w & 3 and part (w - 2) >> 2.  While the K
// loop runs, the epilogue warps already do everything that does not need the
// coupling sums (load theta, its cos and sin, the injection term, the Philox draws
// and Box-Muller noise) and park the results in TMEM columns beside the
// accumulator; once the product is complete only the coupling, the update, the new
// cos / sin and the stores remain.  The warps of a quadrant share its TMEM lanes, so
// each part has its own stash: per 16-column chunk 8 FP32 bases and 8 (cos, sin)
// pairs packed as FP16 (2^-11 relative, far below the BF16 operands' 2^-9).
//
// Tile shapes: 128 columns (10 warps, 3 stages, 97 KB of shared memory, 256 TMEM
// columns: two blocks per SM), 112 columns (the same, with a short second part: more
// tiles, so that the tiles spread over more SMs when 128-wide ones leave SMs with a
// single tile), 256 columns (18 warps, 4 stages, 193 KB, all 512 TMEM columns: one
// block per SM, half the X^T re-reads from L2) and 224 columns (the same block with a
// short last part, 177 KB: nine tile columns of a 2000-node graph fill 144 SMs where
// 256-wide ones fill 128).
template <int BN>
struct TileShape {
    static constexpr int kParts = (BN + 63) / 64;                // 64-column parts (the last may be short)
    static constexpr int kThreads = 64 + 128 * kParts;           // TMA + MMA warps, 4 per part
    static constexpr int kStages = BN <= 128 ? 3 : 4;
    static constexpr int kMinBlocks = BN <= 128 ? 2 : 1;
    static constexpr uint32_t kCols = BN <= 128 ? 256 : 512;      // accumulator, then stashes
    static constexpr uint32_t kStash = kCols / 2;                // part p, chunk k: kStash + 64 p + 16 k
    static constexpr size_t kSmemBytes = (size_t)kStages * (kABytes + BN * 128) + 1024;
    // 16-column chunks of part p
    __host__ __device__ static constexpr int chunks(int p) { return (BN - 64 * p) >= 64 ? 4 : (BN - 64 * p) / 16; }
};

template <int BN>
__global__ void __launch_bounds__(TileShape<BN>::kThreads, TileShape<BN>::kMinBlocks)
    gemm_step_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mW,
                     GemmArgs a) {
    using namespace tc;
    using Sh = TileShape<BN>;
    constexpr int kBN = BN, S = Sh::kStages;
    constexpr uint32_t kCols = Sh::kCols, kStash = Sh::kStash;
    constexpr int kBBytes = kBN * 128;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + S * kABytes;
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int issued, consumed;   // K blocks loaded / multiplied (error-path drain)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int KB = a.n_pad / kBK;
    if (threadIdx.x == 0) {
        issued = 0;
        consumed = 0;
        prefetch_map(&mX);
        prefetch_map(&mW);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // TMA producer: refill a stage as soon as the MMAs reading it have completed
        if (lane == 0) {
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % S;
                if (kb >= S && !mbar_wait(&empty[s], ((kb / S) - 1) & 1, a.err, kErrEmptyWait)) break;
                mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
                tma_load_2d(sA + s * kABytes, &mX, kb * kBK, m0, &full[s]);
                tma_load_2d(sB + s * kBBytes, &mW, kb * kBK, n0, &full[s]);
                issued = kb + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // MMA issuer: waits on data only, so the tensor pipe runs the K loop back to back
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kBM, kBN);
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % S;
                if (!mbar_wait(&full[s], (kb / S) & 1, a.err, kErrFullWait)) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    umma_bf16(tmem, sdesc_kmajor_sw128(a0 + 32 * k), sdesc_kmajor_sw128(b0 + 32 * k), idesc,
                              (kb | k) != 0);
                umma_commit(&empty[s]);
                consumed = kb + 1;
            }
            // completes when every MMA issued above has finished (also after an early exit)
            umma_commit(&done);
        }
        __syncwarp();
    } else {
        const int quad = warp & 3, part = (warp - 2) >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        const int row = m0 + quad * 32 + lane;            // row of X^T: 2 r + comp
        const int r = row >> 1, comp = row & 1;
        const int64_t t = a.t0 ? (int64_t)(*a.t0) + a.t : a.t;
        const float K = __ldg(a.K + t), Ks = __ldg(a.Ks + t), Kn = __ldg(a.Kn + t);
        const float dtK = a.dt * K, dtKs = a.dt * Ks, kick = Kn * a.sqrt_dt;
        float* th_row = a.theta + (size_t)r * a.n_pad;
        const unsigned full_mask = 0xffffffffu;
        const int kChunks = Sh::chunks(part);              // 16-column chunks of this part

        // ---- before the product: per node-replica base = theta - dt Ks sin(2 pi q theta)
        //      + Kn sqrt(dt) xi, and (cos, sin) of theta, parked in TMEM
        // lane pair (cos row, sin row) of replica r: the cos lane finishes nodes 0..7 of
        // each chunk, the sin lane nodes 8..15
#pragma unroll 1
        for (int k = 0; k < kChunks; ++k) {
            const int c0 = part * 64 + 16 * k;
            const int i0 = n0 + c0 + 8 * comp;             // first node of this lane's eight
            float th[8];
            const float4 t0 = *reinterpret_cast<const float4*>(th_row + i0);
            const float4 t1 = *reinterpret_cast<const float4*>(th_row + i0 + 4);
            th[0] = t0.x; th[1] = t0.y; th[2] = t0.z; th[3] = t0.w;
            th[4] = t1.x; th[5] = t1.y; th[6] = t1.z; th[7] = t1.w;
            // Philox blocks: the four replica lanes of a quad that share a half (same comp)
            // need the same block per node; lane rho computes the blocks of nodes rho and
            // rho + 4 of its eight and the group exchanges them by shuffles
            const int rho = (lane >> 1) & 3;
            const uint32_t rq = (uint32_t)(r >> 2);
            const uint64_t seed = *a.seed;
            const uint4 blk0 = draw_block(seed, (uint32_t)a.graph, kStreamNoise, (uint32_t)(i0 + rho),
                                          (uint32_t)t, rq);
            const uint4 blk1 = draw_block(seed, (uint32_t)a.graph, kStreamNoise, (uint32_t)(i0 + rho + 4),
                                          (uint32_t)t, rq);
            uint32_t vb[8], vcs[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int src = (lane & ~7) | ((j & 3) << 1) | comp;
                const uint4 b = (j < 4) ? blk0 : blk1;
                const uint32_t w0 = __shfl_sync(full_mask, b.x, src), w1 = __shfl_sync(full_mask, b.y, src);
                const uint32_t w2 = __shfl_sync(full_mask, b.z, src), w3 = __shfl_sync(full_mask, b.w, src);
                float bj = 0.0f;
                float2 cs = make_float2(0.0f, 0.0f);
                if (i0 + j < a.n) {
                    cs = cos_sin_2pi_fast(th[j]);
                    const float2 zz = (r & 2) ? box_muller_fast(w2, w3) : box_muller_fast(w0, w1);
                    const float z = (r & 1) ? zz.y : zz.x;
                    bj = (th[j] - dtKs * sin_q(a.q, cs.x, cs.y)) + kick * z;
                }
                vb[j] = __float_as_uint(bj);
                const __half2 h = __floats2half2_rn(cs.x, cs.y);
                vcs[j] = *reinterpret_cast<const uint32_t*>(&h);
            }
            const uint32_t col = kStash + 64u * (uint32_t)part + 16u * (uint32_t)k;
            tmem_st8(lane_base + col, vb);
            tmem_st8(lane_base + col + 8, vcs);
        }
        tmem_wait_st();

        // ---- after the product: coupling s A - c B, update, wrap, new (cos, sin)
        // the TMEM loads below are warp-collective: the whole warp goes on, or none of it
        const bool have = __all_sync(full_mask, mbar_wait(&done, 0, a.err, kErrDoneWait));
        tc_fence_after();
        if (have) {
            __nv_bfloat16* xc = a.x_out + (size_t)(2 * r) * a.n_pad;    // cos row of replica r
            __nv_bfloat16* xs = xc + a.n_pad;                              // sin row
#pragma unroll 1
            for (int k = 0; k < kChunks; ++k) {
                const int c0 = part * 64 + 16 * k;
                const int i0 = n0 + c0 + 8 * comp;
                uint32_t v[16], st[16];
                tmem_ld16x2(lane_base + (uint32_t)c0,
                            lane_base + kStash + 64u * (uint32_t)part + 16u * (uint32_t)k, v, st);
                // each lane of the pair needs the other's sums for its eight nodes
                float A[8], B[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float send = __uint_as_float(comp ? v[j] : v[j + 8]);
                    const float recv = __shfl_xor_sync(full_mask, send, 1);
                    A[j] = comp ? recv : __uint_as_float(v[j]);
                    B[j] = comp ? __uint_as_float(v[j + 8]) : recv;
                }
                float th[8];
                __align__(16) __nv_bfloat16 oc[8], os[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t hw = st[8 + j];
                    const float2 cs = __half22float2(*reinterpret_cast<const __half2*>(&hw));
                    const float d = cs.y * A[j] - cs.x * B[j];
                    const float tn = (i0 + j < a.n) ? wrap01(__uint_as_float(st[j]) + dtK * d) : 0.0f;
                    const float2 ncs = (i0 + j < a.n) ? cos_sin_2pi_fast(tn) : make_float2(0.0f, 0.0f);
                    th[j] = tn;
                    oc[j] = __float2bfloat16_rn(ncs.x);
                    os[j] = __float2bfloat16_rn(ncs.y);
                }
                *reinterpret_cast<float4*>(th_row + i0) = make_float4(th[0], th[1], th[2], th[3]);
                *reinterpret_cast<float4*>(th_row + i0 + 4) = make_float4(th[4], th[5], th[6], th[7]);
                *reinterpret_cast<uint4*>(xc + i0) = *reinterpret_cast<const uint4*>(oc);
                *reinterpret_cast<uint4*>(xs + i0) = *reinterpret_cast<const uint4*>(os);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a timed-out wait, let copies still in flight land before the block exits
    if (threadIdx.x == 0)
        for (int kb = consumed; kb < issued; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1, a.err, kErrFullWait);
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ----------------------------------------------------------------------------- set-up
__global__ void gemm_init_kernel(int n, int n_pad, int R_pad, const uint64_t* seed_dev, int graph, float* theta,
                                 __nv_bfloat16* x) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)R_pad * n_pad) return;
    const int r = (int)(gid / n_pad), i = (int)(gid - (int64_t)r * n_pad);
    float th = 0.0f, c = 0.0f, s = 0.0f;
    if (i < n) {
        const uint4 w = draw_block(*seed_dev, (uint32_t)graph, kStreamInit, (uint32_t)i, 0, (uint32_t)(r >> 2));
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        th = u01(words[r & 3]);
        const float2 cs = cos_sin_2pi_fast(th);
        c = cs.x;
        s = cs.y;
    }
    theta[gid] = th;
    x[(size_t)(2 * r) * n_pad + i] = __float2bfloat16_rn(c);
    x[(size_t)(2 * r + 1) * n_pad + i] = __float2bfloat16_rn(s);
}

// dense W[i][j] = w_ij (zero elsewhere, including the padding)
__global__ void gemm_scatter_kernel(CSRDev csr, int g, int n_pad, __nv_bfloat16* W) {
    const GraphDev gd = csr.graphs[g];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gd.n) return;
    const int node = gd.node_off + i;
    for (int e = csr.rowp[node]; e < csr.rowp[node + 1]; ++e) {
        const uint32_t cw = csr.col[e];
        const int j = (int)checked_node(csr, g, csr.w ? cw : (cw & ~kSignBit), (uint32_t)node) - gd.node_off;
        const float w = csr.w ? csr.w[e] : ((cw & kSignBit) ? -1.0f : 1.0f);
        W[(size_t)i * n_pad + j] = __float2bfloat16_rn(w);
    }
}

// theta [R_pad][n_pad] -> the common [node][R_pad] layout (for readout)
__global__ void gemm_to_common_kernel(int n, int n_pad, int R_pad, int node_off, const float* theta,
                                      float* out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * R_pad) return;
    const int i = (int)(gid / R_pad), r = (int)(gid - (int64_t)i * R_pad);
    out[(size_t)(node_off + i) * R_pad + r] = theta[(size_t)r * n_pad + i];
}

// ---------------------------------------------------------------- readout on tensor cores
// X^T rows 2r and 2r + 1 = the spins s_r = +-1 of replica r (BF16, exact), 0 beyond n.
__global__ void gemm_spins_kernel(int n, int n_pad, int R_pad, const float* __restrict__ theta,
                                  __nv_bfloat16* __restrict__ x) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)R_pad * n_pad) return;
    const int r = (int)(gid / n_pad), i = (int)(gid - (int64_t)r * n_pad);
    const float sgn = i < n ? (spin_of(theta[gid], 2) ? -1.0f : 1.0f) : 0.0f;
    x[(size_t)(2 * r) * n_pad + i] = __float2bfloat16_rn(sgn);
    x[(size_t)(2 * r + 1) * n_pad + i] = __float2bfloat16_rn(sgn);
}

// The agreeing weight of every replica of one dense graph from P^T = X^T W with the spin
// rows above: a 128 x 128 tile of P^T (64 replicas x 128 nodes) per block, one thread
// streaming the K blocks with TMA and issuing tcgen05.mma into TMEM, then each thread of
// an even X^T row (replica r) sums s_{r,c} P[r][c] over the tile's 128 columns (integers,
// exact in FP32) and adds a quarter of it, FP64, to agree[r]; the block of the first
// column tile also adds a quarter of sum_ij w_ij.  sum_{i<j} w_ij [s_i == s_j] =
// (sum_ij w_ij + s^T W s) / 4.  Bounded waits as in the step kernel.
struct ScoreArgs {
    const float* theta;      // [R_pad][n_pad] phases (the spins' source, for s_{r,c})
    double* agree;           // [G][row_stride][R_pad]
    int64_t row_stride, k;   // readout slot k, or from the device step base
    const int32_t* t0;
    int32_t t_add, every;
    int32_t graph, n_pad, R, R_pad;
    double wsum4;            // sum_ij w_ij / 4
    int32_t* err;
};

__global__ void __launch_bounds__(128, 1)
    gemm_score_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mW, ScoreArgs a) {
    using namespace tc;
    constexpr int S = 4, kBN = 128, kBBytes = kBN * 128;
    constexpr uint32_t kCols = 128;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + S * kABytes;
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int KB = a.n_pad / kBK;
    if (threadIdx.x == 0) {
        prefetch_map(&mX);
        prefetch_map(&mW);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16_f32(kBM, kBN);
        int pending[S];
        auto load = [&](int kb) {
            const int s = kb % S;
            mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
            tma_load_2d(sA + s * kABytes, &mX, kb * kBK, m0, &full[s]);
            tma_load_2d(sB + s * kBBytes, &mW, kb * kBK, n0, &full[s]);
            pending[s] = kb;
        };
        for (int s = 0; s < S; ++s) pending[s] = -1;
        for (int kb = 0; kb < KB && kb < S; ++kb) load(kb);
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % S;
            if (!mbar_wait(&full[s], (kb / S) & 1, a.err, kErrFullWait)) break;
            pending[s] = -1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                umma_bf16(tmem, sdesc_kmajor_sw128(a0 + 32 * k), sdesc_kmajor_sw128(b0 + 32 * k), idesc,
                          (kb | k) != 0);
            umma_commit(&empty[s]);
            if (kb + S < KB) {
                if (!mbar_wait(&empty[s], (kb / S) & 1, a.err, kErrEmptyWait)) break;
                load(kb + S);
            }
        }
        // loads still in flight after a wait that gave up land before the block exits
        for (int s = 0; s < S; ++s)
            if (pending[s] >= 0) mbar_wait(&full[s], (pending[s] / S) & 1, a.err, kErrFullWait);
        umma_commit(&done);
    }
    __syncwarp();
    const bool have = __all_sync(0xffffffffu, mbar_wait(&done, 0, a.err, kErrDoneWait));
    tc_fence_after();
    if (have) {
        const int row = m0 + warp * 32 + lane;   // X^T row; even rows carry replica row / 2
        const int r = row >> 1;
        const float* th = a.theta + (size_t)r * a.n_pad + n0;
        float p = 0.0f;
#pragma unroll 1
        for (int c = 0; c < kBN; c += 16) {
            if (n0 + c >= a.n_pad) break;   // the last tile may reach past n_pad (a multiple of 64)
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
                const float4 t4 = *reinterpret_cast<const float4*>(th + c + j);
                const float tt[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // columns beyond n hold spin 0 in X^T and zero rows of W: P is 0 there
                    const float sg = spin_of(tt[u], 2) ? -1.0f : 1.0f;
                    p = __fmaf_rn(sg, __uint_as_float(v[j + u]), p);
                }
            }
        }
        if ((row & 1) == 0 && r < a.R) {
            const int64_t k = a.t0 ? ((int64_t)(*a.t0) + a.t_add) / a.every - 1 : a.k;
            double* dst = a.agree + ((int64_t)a.graph * a.row_stride + k) * a.R_pad + r;
            atomicAdd(dst, 0.25 * (double)p + (blockIdx.x == 0 ? a.wsum4 : 0.0));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

}  // namespace

// 128-wide tiles with three stages use 97 KB of shared memory and 256 TMEM columns,
// so two blocks share an SM (and its 512 TMEM columns).
// Tile width of the dense form.  threads_per_block 576 asks for one block per SM with
// 224- or 256-wide tiles; 320 for two blocks per SM with 112- or 128-wide ones; 0 takes
// the wide tiles for graphs of 3000 nodes or more (measured: 4-5 % faster at n = 4000;
// at n = 2000, 224-wide tiles 19.9 against 20.4 us/step with 1024 replicas and equal
// with 4096; the autotuner times both block sizes).  Within each pair the width whose
// busiest SM carries the fewest tile columns wins, the wider on a tie (fewer X^T
// re-reads).
int gemm_bn_for(const oim_run_s& r, int n) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        sms = (cudaGetDevice(&dev) == cudaSuccess &&
               cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
                  ? v
                  : 152;
    }
    const int64_t mt = (2 * (int64_t)r.R_pad) / kBM;
    // tile columns on the busiest SM with `per_sm` blocks an SM
    auto cost = [&](int bn, int per_sm) {
        const int64_t tiles = (int64_t)((n + bn - 1) / bn) * mt;
        return ((tiles + (int64_t)sms * per_sm - 1) / ((int64_t)sms * per_sm)) * per_sm * bn;
    };
    if (r.opts.threads_per_block == TileShape<256>::kThreads || (r.opts.threads_per_block == 0 && n >= 3000))
        return cost(224, 1) < cost(256, 1) ? 224 : 256;
    return cost(112, 2) < cost(128, 2) ? 112 : 128;
}

constexpr size_t kScoreSmem = 4 * (size_t)(kABytes + 128 * 128) + 1024;

// Device state of the dense form for graph `graph` of the problem, appended to
// oim_run_s::gemms (the dense form's one graph, or a dense member of a mixed run).
int gemm_setup(oim_run_s& r, int graph) {
    const GraphDev& gd = r.p->graphs[graph];
    r.gemms.emplace_back();
    GemmState& st = r.gemms.back();
    st.graph = graph;
    st.n = gd.n;
    st.bn = gemm_bn_for(r, gd.n);
    st.tiles_n = (gd.n + st.bn - 1) / st.bn;
    // row length and K extent: the tiles' columns, rounded up to the 64-wide K blocks
    st.n_pad = ((st.tiles_n * st.bn + kBK - 1) / kBK) * kBK;
    const size_t nth = (size_t)r.R_pad * st.n_pad;
    cudaError_t e = cudaMalloc(&st.theta, nth * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&st.x[0], 2 * nth * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&st.x[1], 2 * nth * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&st.w, (size_t)st.n_pad * st.n_pad * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(dense form)");
    e = cudaMemset(st.w, 0, (size_t)st.n_pad * st.n_pad * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(st.x[1], 0, 2 * nth * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(dense form)");
    gemm_scatter_kernel<<<(gd.n + 255) / 256, 256>>>(r.p->csr(), graph, st.n_pad,
                                                     reinterpret_cast<__nv_bfloat16*>(st.w));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dense coupling matrix");
    int rc = make_map_bf16(&st.map_w, st.w, st.n_pad, st.n_pad, (uint64_t)st.n_pad * 2, st.bn);
    if (rc == OIM_OK) rc = make_map_bf16(&st.map_w128, st.w, st.n_pad, st.n_pad, (uint64_t)st.n_pad * 2, 128);
    // readouts on the tensor cores when every weight of the graph is exact in BF16
    // (and every partial sum an integer below 2^24: 128 columns of row sums below 2^17)
    st.score_tc = r.p->q == 2;
    for (int32_t i = 0; i < gd.n && st.score_tc; ++i) {
        const int32_t v = gd.node_off + i;
        double row = 0.0;
        for (int64_t e = r.p->h_rowp[(size_t)v]; e < r.p->h_rowp[(size_t)v + 1]; ++e) {
            const float x = r.p->h_w[(size_t)e];
            if (x != std::floor(x) || std::fabs(x) > 256.0f) st.score_tc = false;
            row += std::fabs((double)x);
        }
        if (row >= 131072.0) st.score_tc = false;
    }
    for (int b = 0; b < 2 && rc == OIM_OK; ++b)
        rc = make_map_bf16(&st.map_x[b], st.x[b], st.n_pad, 2 * (uint64_t)r.R_pad, (uint64_t)st.n_pad * 2, 128);
    if (rc != OIM_OK) return rc;
    // opt in to the large shared-memory footprint once, outside any stream capture
    e = cudaFuncSetAttribute(gemm_step_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TileShape<128>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_step_kernel<112>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TileShape<112>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_step_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TileShape<256>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_step_kernel<224>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TileShape<224>::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScoreSmem);
    if (e != cudaSuccess) return cuda_fail(e, "dense form shared memory");
    return OIM_OK;
}

void gemm_free(oim_run_s& r) {
    for (GemmState& st : r.gemms) {
        cudaFree(st.theta);
        cudaFree(st.x[0]);
        cudaFree(st.x[1]);
        cudaFree(st.w);
    }
    r.gemms.clear();
}

StepParams make_params(const oim_run_s& r);

cudaError_t launch_gemm_init(const oim_run_s& r, int k, cudaStream_t s) {
    const GemmState& st = r.gemms[k];
    const int64_t total = (int64_t)r.R_pad * st.n_pad;
    gemm_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        st.n, st.n_pad, r.R_pad, r.d_seed, st.graph, st.theta, reinterpret_cast<__nv_bfloat16*>(st.x[0]));
    return cudaGetLastError();
}

// Step t of dense state k.  With d_t0 the step is *d_t0 + t (t the offset in a replayed
// chunk, whose parity is the step's: chunks have an even length).
cudaError_t launch_gemm_step_at(const oim_run_s& r, int k, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    const GemmState& st = r.gemms[k];
    const StepParams P = make_params(r);
    const size_t soff = (size_t)st.graph * P.steps;   // the graph's row of the schedules
    GemmArgs a;
    a.theta = st.theta;
    a.x_out = reinterpret_cast<__nv_bfloat16*>(st.x[(t + 1) & 1]);
    a.K = P.K + soff;
    a.Ks = P.Ks + soff;
    a.Kn = P.Kn + soff;
    a.t = t;
    a.t0 = d_t0;
    a.dt = P.dt;
    a.sqrt_dt = P.sqrt_dt;
    a.seed = r.d_seed;
    a.graph = st.graph;
    a.q = P.q;
    a.n = st.n;
    a.n_pad = st.n_pad;
    a.err = r.d_err;
    const dim3 grid(st.tiles_n, (2 * r.R_pad) / kBM);
    if (st.bn == 256)
        gemm_step_kernel<256><<<grid, TileShape<256>::kThreads, TileShape<256>::kSmemBytes, s>>>(
            st.map_x[t & 1], st.map_w, a);
    else if (st.bn == 224)
        gemm_step_kernel<224><<<grid, TileShape<224>::kThreads, TileShape<224>::kSmemBytes, s>>>(
            st.map_x[t & 1], st.map_w, a);
    else if (st.bn == 112)
        gemm_step_kernel<112><<<grid, TileShape<112>::kThreads, TileShape<112>::kSmemBytes, s>>>(
            st.map_x[t & 1], st.map_w, a);
    else
        gemm_step_kernel<128><<<grid, TileShape<128>::kThreads, TileShape<128>::kSmemBytes, s>>>(
            st.map_x[t & 1], st.map_w, a);
    return cudaGetLastError();
}

// The agreeing weight of dense state k's replicas into readout slot k_slot (or the slot
// of the device step base), on the tensor cores: the spins into X^T buffer xbuf (the one
// the next step does not read), then P^T = X^T W.  Requires st.score_tc.
cudaError_t launch_gemm_score(const oim_run_s& r, int k, int64_t k_slot, const int32_t* d_t0, int32_t t_add,
                              int xbuf, cudaStream_t s) {
    const GemmState& st = r.gemms[k];
    const int64_t total = (int64_t)r.R_pad * st.n_pad;
    gemm_spins_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        st.n, st.n_pad, r.R_pad, st.theta, reinterpret_cast<__nv_bfloat16*>(st.x[xbuf]));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ScoreArgs a;
    a.theta = st.theta;
    a.agree = r.d_trace;
    a.row_stride = r.readouts_cap;
    a.k = k_slot;
    a.t0 = d_t0;
    a.t_add = t_add;
    a.every = (int32_t)std::max<int64_t>(1, r.readout_every);
    a.graph = st.graph;
    a.n_pad = st.n_pad;
    a.R = r.R;
    a.R_pad = r.R_pad;
    a.wsum4 = 0.5 * r.p->graphs[st.graph].wtot;   // sum_ij w_ij / 4 = 2 wtot / 4
    a.err = r.d_err;
    const dim3 grid((unsigned)((st.n_pad + 127) / 128), (unsigned)((2 * r.R_pad) / kBM));
    gemm_score_kernel<<<grid, 128, kScoreSmem, s>>>(st.map_x[xbuf], st.map_w128, a);
    return cudaGetLastError();
}

// dense state k's phases into `out` in the common [node][R_pad] layout
cudaError_t launch_gemm_to_common(const oim_run_s& r, int k, float* out, cudaStream_t s) {
    const GemmState& st = r.gemms[k];
    const int64_t total = (int64_t)st.n * r.R_pad;
    gemm_to_common_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        st.n, st.n_pad, r.R_pad, r.p->graphs[st.graph].node_off, st.theta, out);
    return cudaGetLastError();
}

}  // namespace oim

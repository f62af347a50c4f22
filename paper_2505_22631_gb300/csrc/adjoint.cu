// adjoint.cu -- gradients of the relaxed energy with respect to the schedules.
//
// Loss of graph g: L_g = (1/R) sum_r E_g(theta_T^r), E of Eq. 6 on the final
// phases.  The forward map of one step (Algorithm 1, Eq. 5) is
//   theta_{t+1} = wrap(theta_t + dt f(theta_t; K_t, Ks_t) + Kn_t sqrt(dt) xi_t),
// whose wrap has unit derivative (every function of the phases is 1-periodic).
// With lambda_t = dL/dtheta_t:
//   lambda_T   = -(2 pi / R) D(theta_T),  D_i = sum_j w_ij sin 2 pi (theta_i - theta_j)
//   lambda_t,j = lambda_{t+1,j} + dt [ lambda_{t+1,j} (2 pi K_t S_j - 2 pi q Ks_t cos 2 pi q theta_j)
//                                      - 2 pi K_t C_j ]
//   S_j = sum_k w_jk cos 2 pi (theta_j - theta_k) = c_j A_j + s_j B_j
//   C_j = sum_k w_jk lambda_{t+1,k} cos 2 pi (theta_k - theta_j) = c_j P_j + s_j Q_j
// where (A, B, P, Q)_j = sum_k w_jk (c_k, s_k, lambda_k c_k, lambda_k s_k), all at theta_t.
// Schedule gradients, summed over nodes and replicas of each graph (the terms of a warp,
// at most 128, in FP32 -- a relative error of ~1e-5 of their absolute sum, far inside the
// adjoint's FP32 tolerance -- and the warps' sums in FP64):
//   dL/dK_t = dt sum lambda_{t+1} D(theta_t),  dL/dKs_t = -dt sum lambda_{t+1} sin 2 pi q theta_t,
//   dL/dKn_t = sqrt(dt) sum lambda_{t+1} xi_t  (pathwise: the same Philox draws as the forward).
// Layout as the stream form: [node][R_pad], replicas contiguous, a thread per (node, quad).
// The forward recomputation of a segment keeps the coupling sums (A, B) of each of its
// steps (the forward step computes them anyway), so the reverse sweep gathers only the
// two planes lambda_{t+1} c_t and lambda_{t+1} s_t of [node][R_pad] floats (two 16-byte
// loads per neighbour that a warp turns into whole 512-byte rows).  Each adjoint step
// also writes the planes the next one (step t - 1) gathers, lambda_t (c, s)_{t-1}, from
// its own lambda_t and theta_{t-1}.
#include "oim_checks.cuh"
#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {

namespace {

constexpr float kTwoPi = 6.28318530717958647f;

// (c, s) of every node-replica at theta as two planes, or (lambda c, lambda s) when lam
// is given.
__global__ void __launch_bounds__(256) adj_planes_kernel(int64_t state, const float* __restrict__ theta,
                                                         const float* __restrict__ lam, float* __restrict__ Y) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= state) return;
    float s, c;
    if (lam) {   // lambda planes, as the adjoint step writes them (hardware sin / cos)
        const float2 cs = cos_sin_2pi_fast(theta[gid]);
        c = cs.x;
        s = cs.y;
    } else {     // (c, s) of the final phases for the terminal adjoint and the loss
        sincospif(2.0f * theta[gid], &s, &c);
    }
    const float l = lam ? lam[gid] : 1.0f;
    Y[gid] = lam ? l * c : c;
    Y[state + gid] = lam ? l * s : s;
}

// D(theta) * scale into lam (the terminal adjoint, scale = -2 pi / R), and the
// per-graph FP64 sum of E = 1/2 sum_i (c_i A_i + s_i B_i) over the real replicas.
// Y: the (c, s) planes of theta.
__global__ void __launch_bounds__(128) adj_terminal_kernel(CSRDev csr, int R, int R_pad, float scale,
                                                           const float* __restrict__ Y,
                                                           float* __restrict__ lam,
                                                           double* __restrict__ loss) {
    const int quads = R_pad >> 2;
    const int node = blockIdx.x * blockDim.y + threadIdx.y;   // block: quads x nodes
    const int quad = blockIdx.y * blockDim.x + threadIdx.x;
    double e = 0.0;
    int g = -1;
    if (node < csr.nodes && quad < quads) {
        g = csr.node_graph[node];
        const size_t at = (size_t)node * R_pad + 4 * quad;
        const size_t state = (size_t)csr.nodes * R_pad;
        const float* Yc = Y;
        const float* Ys = Y + state;
        float A[4] = {0, 0, 0, 0}, B[4] = {0, 0, 0, 0};
        for (int ei = csr.rowp[node]; ei < csr.rowp[node + 1]; ++ei) {
            const uint32_t cw = csr.col[ei];
            const uint32_t j = checked_node_of_row(csr, node, csr.w ? cw : (cw & ~kSignBit));
            const float w = csr.w ? csr.w[ei] : ((cw & kSignBit) ? -1.0f : 1.0f);
            const size_t jat = (size_t)j * R_pad + 4 * quad;
            const float4 c4 = *reinterpret_cast<const float4*>(Yc + jat);
            const float4 s4 = *reinterpret_cast<const float4*>(Ys + jat);
            const float cj[4] = {c4.x, c4.y, c4.z, c4.w}, sj[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                A[v] = fmaf(w, cj[v], A[v]);
                B[v] = fmaf(w, sj[v], B[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float c = Yc[at + v], sn = Ys[at + v];
            lam[at + v] = scale * (sn * A[v] - c * B[v]);
            if (4 * quad + v < R) e += 0.5 * (double)(c * A[v] + sn * B[v]);
        }
    }
    // block reduce per graph: blocks may straddle graphs, so reduce by atomics per thread group
    if (g >= 0 && e != 0.0) atomicAdd(loss + g, e);
}

// One adjoint step: lambda_out = lambda_t from lambda_in = lambda_{t+1} at theta_t,
// the step's gradient terms added to dK[g][t], dKs[g][t], dKn[g][t], and, when
// theta_prev (theta_{t-1}) is given, the planes lambda_t (c, s)_{t-1} for step t - 1.
//   AB   the forward step's coupling sums at theta_t, float2 [node][R_pad]
//   Ylam the planes lambda_{t+1} c_t, lambda_{t+1} s_t
// 64 registers, 32 warps per SM (measured: 726 -> 699 ms for the backward pass of the
// schedule workload against the unbounded 70 registers)
__global__ void __launch_bounds__(128, 8) adj_step_kernel(CSRDev csr, StepParams P, int64_t t,
                                                       const float* __restrict__ theta,
                                                       const float* __restrict__ theta_prev,
                                                       const float2* __restrict__ AB,
                                                       const float* __restrict__ Ylam,
                                                       float* __restrict__ Ylam_out,
                                                       const float* __restrict__ lam_in,
                                                       float* __restrict__ lam_out,
                                                       double* __restrict__ dK, double* __restrict__ dKs,
                                                       double* __restrict__ dKn, int64_t T,
                                                       int quads_fast) {
    // block: quads x nodes; the blocks take their nodes graph by graph, heaviest row
    // first within a graph (so a warp's nodes share a graph for the gradient
    // reductions), with the replica blocks dispatched first under quads_fast
    const int quads = P.R_pad >> 2;
    const int nblk = quads_fast ? blockIdx.y : blockIdx.x;
    const int qblk = quads_fast ? blockIdx.x : blockIdx.y;
    const int slot = nblk * blockDim.y + threadIdx.y;
    const int quad = qblk * blockDim.x + threadIdx.x;
    const bool valid = slot < csr.nodes && quad < quads;   // no early exit: the warp shuffles below
    int g = -1;
    // gradient terms: a warp's (at most 128) in FP32, the warps' sums in FP64 atomics
    float gK = 0.f, gS = 0.f, gN = 0.f;
    if (valid) {
        const int4 row = __ldg(csr.arow + slot);   // {node, row start, first -1 entry, row end}
        const int node = row.x;
        const size_t at = (size_t)node * P.R_pad + 4 * quad;
        const size_t state = (size_t)csr.nodes * P.R_pad;
        const float* Ylc = Ylam;
        const float* Yls = Ylam + state;
        float Pp[4] = {0, 0, 0, 0}, Q[4] = {0, 0, 0, 0};
        for (int ei = row.y; ei < row.w; ++ei) {
            const uint32_t cw = csr.col[ei];
            const uint32_t j = checked_node_of_row(csr, node, csr.w ? cw : (cw & ~kSignBit));
            const float w = csr.w ? csr.w[ei] : ((cw & kSignBit) ? -1.0f : 1.0f);
            const size_t jat = (size_t)j * P.R_pad + 4 * quad;
            const float4 lc4 = *reinterpret_cast<const float4*>(Ylc + jat);
            const float4 ls4 = *reinterpret_cast<const float4*>(Yls + jat);
            const float lcj[4] = {lc4.x, lc4.y, lc4.z, lc4.w}, lsj[4] = {ls4.x, ls4.y, ls4.z, ls4.w};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                Pp[v] = fmaf(w, lcj[v], Pp[v]);
                Q[v] = fmaf(w, lsj[v], Q[v]);
            }
        }
        // the node's own values after the gather: only the gather's state is live during it
        g = csr.node_graph[node];
        const int i = node - csr.graphs[g].node_off;
        const size_t sidx = (size_t)g * P.steps + t;
        const float K = P.K[sidx], Ks = P.Ks[sidx];
        const uint4 x = draw_block(P.seed_dev ? *P.seed_dev : P.seed, (uint32_t)g, kStreamNoise, (uint32_t)i, (uint32_t)t,
                                   (uint32_t)quad);
        // the per-step terms take the hardware sin / cos / log2 / sqrt (absolute errors
        // ~1e-6, three orders below the adjoint's FP32 tolerance against FP64)
        const float2 z01 = box_muller_fast(x.x, x.y);
        const float2 z23 = box_muller_fast(x.z, x.w);
        const float z[4] = {z01.x, z01.y, z23.x, z23.y};
        const float4 ab01 = *reinterpret_cast<const float4*>(AB + at);
        const float4 ab23 = *reinterpret_cast<const float4*>(AB + at + 2);
        const float A[4] = {ab01.x, ab01.z, ab23.x, ab23.z}, B[4] = {ab01.y, ab01.w, ab23.y, ab23.w};
        float lt[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float th = theta[at + v];
            const float2 cs1 = cos_sin_2pi_fast(th);
            const float c = cs1.x, s = cs1.y;
            const float l = lam_in[at + v];
            const float S = c * A[v] + s * B[v];
            const float Cc = c * Pp[v] + s * Q[v];
            const float qth = (float)P.q * th;
            const float2 csq = cos_sin_2pi_fast(qth - floorf(qth));
            const float sq = csq.y, cq = csq.x;
            const float diag = kTwoPi * K * S - kTwoPi * (float)P.q * Ks * cq;
            lt[v] = l + P.dt * (l * diag - kTwoPi * K * Cc);
            lam_out[at + v] = lt[v];
            if (4 * quad + v < P.R) {
                const float D = s * A[v] - c * B[v];
                gK = fmaf(l, D, gK);
                gS = fmaf(l, sq, gS);
                gN = fmaf(l, z[v], gN);
            }
        }
        if (theta_prev) {
            // the planes step t - 1 gathers: lambda_t (c, s) of theta_{t-1}
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float2 cs0 = cos_sin_2pi_fast(theta_prev[at + v]);
                Ylam_out[at + v] = lt[v] * cs0.x;
                Ylam_out[state + at + v] = lt[v] * cs0.y;
            }
        }
    }
    // warp reduction when every lane belongs to the same graph, else per-lane atomics
    const unsigned full = 0xffffffffu;
    const int g0 = __shfl_sync(full, g, 0);
    if (__all_sync(full, g == g0)) {
        for (int m = 16; m >= 1; m >>= 1) {
            gK += __shfl_xor_sync(full, gK, m);
            gS += __shfl_xor_sync(full, gS, m);
            gN += __shfl_xor_sync(full, gN, m);
        }
        const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;   // warps run over the linear index
        if (lane != 0 || g < 0) return;
    } else if (g < 0) {
        return;
    }
    atomicAdd(dK + (size_t)g * T + t, (double)P.dt * (double)gK);
    atomicAdd(dKs + (size_t)g * T + t, -(double)P.dt * (double)gS);
    atomicAdd(dKn + (size_t)g * T + t, (double)P.sqrt_dt * (double)gN);
}

}  // namespace

StepParams make_params(const oim_run_s& r);

// Blocks of 128 threads: x over replica quads (a warp covers consecutive quads of a
// node), y over nodes; the grid runs nodes along x and quads along y.  (Against blocks of
// 256: the backward pass of the 64-graph schedule workload 237.1 -> 230.3 ms, a block's
// slot freeing as soon as its fewer nodes are done.)
struct QuadGridA {
    dim3 grid, block;
};
static QuadGridA quad_grid_a(int64_t nodes, int quads) {
    int qx = 1;
    while (qx < quads && qx < 32) qx <<= 1;
    const int ny = 128 / qx;
    QuadGridA q;
    q.block = dim3((unsigned)qx, (unsigned)ny);
    q.grid = dim3((unsigned)((nodes + ny - 1) / ny), (unsigned)((quads + qx - 1) / qx));
    return q;
}

// Two planes of [node][R_pad] floats from theta: (c, s), or (lambda c, lambda s).
cudaError_t launch_adj_planes(const oim_run_s& r, const float* theta, const float* lam, float* Y,
                              cudaStream_t s) {
    const int64_t total = r.p->nodes * r.R_pad;
    adj_planes_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, theta, lam, Y);
    return cudaGetLastError();
}

// lambda_T and the loss sums from the (c, s) planes of theta_T.
cudaError_t launch_adj_terminal(const oim_run_s& r, const float* Y, float* lam, double* loss,
                                cudaStream_t s) {
    const float scale = -6.28318530717958647f / (float)r.R;
    const QuadGridA q = quad_grid_a(r.p->nodes, r.R_pad / 4);
    adj_terminal_kernel<<<q.grid, q.block, 0, s>>>(r.p->csr(), r.R, r.R_pad, scale, Y, lam, loss);
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const oim_run_s& r, int64_t t, const float* theta, const float* theta_prev,
                            const float2* AB, const float* Ylam, float* Ylam_out, const float* lam_in,
                            float* lam_out, double* dK, double* dKs, double* dKn, cudaStream_t s) {
    const StepParams P = make_params(r);
    QuadGridA q = quad_grid_a(r.p->nodes, r.R_pad / 4);
    int quads_fast = 0;
    if (q.grid.x <= 65535u) {   // node blocks along y, replica blocks along x
        q.grid = dim3(q.grid.y, q.grid.x);
        quads_fast = 1;
    }
    adj_step_kernel<<<q.grid, q.block, 0, s>>>(r.p->csr(), P, t, theta, theta_prev, AB, Ylam, Ylam_out, lam_in,
                                               lam_out, dK, dKs, dKn, r.steps, quads_fast);
    return cudaGetLastError();
}

}  // namespace oim

// readout.cu -- phase threshold, cut / conflict scores and the Eq. 6 energy.
//
// The paper's phase threshold kernel maps each phase to the nearest stable
// phase k/q (Sec. III-B); the score of a spin assignment is the cut weight
// (Ising max-cut, Eq. 1) or the weight of monochromatic edges (Potts colouring,
// Eq. 2).  Scores are accumulated as the weight of agreeing edges,
// sum_{i<j} w_ij [s_i == s_j], in FP64; the cut is wtot - agree.  With integer
// weights every partial sum is an integer below 2^53, so the result is exact
// whatever the order of the additions.
#include <algorithm>
#include <type_traits>

#include "oim_checks.cuh"
#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {

namespace {

// Spins of every (node, replica) for the score pass: spins[node][R_pad] =
// floor(q theta + 1/2) mod q (the FP32 decision of spin_of), four replicas a thread.
__global__ void __launch_bounds__(256) spin_kernel(const float* __restrict__ theta, int64_t quads, int q,
                                                   int8_t* __restrict__ spins) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= quads) return;
    const float4 t = reinterpret_cast<const float4*>(theta)[gid];
    reinterpret_cast<char4*>(spins)[gid] =
        make_char4((signed char)spin_of(t.x, q), (signed char)spin_of(t.y, q), (signed char)spin_of(t.z, q),
                   (signed char)spin_of(t.w, q));
}

// Block = 32 replica quads x 8 node lanes; it owns a chunk of 8 * npt consecutive
// nodes, lane y taking nodes y, y + 8, ...  Each thread sums, for its four replicas,
// the agreeing weight of its nodes' upper-triangle entries (j > i, a separate CSR in
// row order) from the spins, four entries at a time so that four gathers are in
// flight.  When the chunk lies in one graph the eight lanes are summed in shared
// memory and one FP64 atomic per replica and block goes out (thousands of blocks
// adding into the same few replica sums is what limits the pass otherwise); a chunk
// that straddles graphs flushes per thread at each graph change.
constexpr int kScoreQuads = 32, kScoreLanes = 8;

// kF32: the thread's running sums in FP32 (launched for +-1 weights when npt x the
// largest row length stays below 2^24, so every partial sum is an integer exact in FP32;
// FP64 arithmetic is slow on this part), else in FP64.
template <bool kF32>
__global__ void __launch_bounds__(kScoreQuads * kScoreLanes) score_kernel(
    CSRDev csr, const int8_t* __restrict__ spins, int R_pad, double* __restrict__ agree, int64_t row_stride,
    int64_t k_fixed, int npt, const int32_t* __restrict__ d_t0, int32_t t_add, int32_t every, int node_lo,
    int node_hi) {
    __shared__ double red[kScoreLanes][kScoreQuads][4];
    // readout slot: fixed, or (in a replayed chunk of steps) from the device step base
    const int64_t k = d_t0 ? ((int64_t)(*d_t0) + t_add) / every - 1 : k_fixed;
    const int quads = R_pad >> 2;
    const int quad = blockIdx.x * kScoreQuads + threadIdx.x;
    const bool valid = quad < quads;      // no early exit: the block synchronises below
    const int chunk0 = node_lo + blockIdx.y * kScoreLanes * npt;
    const int chunk1 = min(chunk0 + kScoreLanes * npt, node_hi);
    const bool one_graph = csr.node_graph[chunk0] == csr.node_graph[chunk1 - 1];
    const char4* sp = reinterpret_cast<const char4*>(spins) + (valid ? quad : 0);
    using Acc = typename std::conditional<kF32, float, double>::type;
    Acc acc[4] = {0, 0, 0, 0};
    int g_cur = -1;
    auto flush = [&]() {
        if (g_cur < 0) return;
        double* dst = agree + ((int64_t)g_cur * row_stride + k) * R_pad + 4 * quad;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (acc[c] != 0) atomicAdd(dst + c, (double)acc[c]);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = 0;
    };
    for (int node = chunk0 + threadIdx.y; valid && node < chunk1; node += kScoreLanes) {
        const int g = csr.node_graph[node];
        if (g != g_cur) {
            if (!one_graph) flush();
            g_cur = g;
        }
        const char4 si = sp[(size_t)node * quads];
        // per node the sum has at most max_deg terms; FP32 is exact for integer w
        // below 2^24 / max_deg and close otherwise, the FP64 sum carries it on
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
        auto add = [&](uint32_t cw, float wv, char4 sj) {
            const float w = csr.uw ? wv : ((cw & kSignBit) ? -1.0f : 1.0f);
            f0 += (si.x == sj.x) ? w : 0.f;
            f1 += (si.y == sj.y) ? w : 0.f;
            f2 += (si.z == sj.z) ? w : 0.f;
            f3 += (si.w == sj.w) ? w : 0.f;
        };
        auto row_of = [&](uint32_t cw) {
            return sp[(size_t)checked_node_of_row(csr, node, csr.uw ? cw : (cw & ~kSignBit)) * quads];
        };
        const int e_end = csr.urowp[node + 1];
        int e = csr.urowp[node];
        for (; e + 4 <= e_end; e += 4) {
            const uint32_t c0 = csr.ucol[e], c1 = csr.ucol[e + 1], c2 = csr.ucol[e + 2], c3 = csr.ucol[e + 3];
            const char4 s0 = row_of(c0), s1 = row_of(c1), s2 = row_of(c2), s3 = row_of(c3);
            add(c0, csr.uw ? csr.uw[e] : 0.f, s0);
            add(c1, csr.uw ? csr.uw[e + 1] : 0.f, s1);
            add(c2, csr.uw ? csr.uw[e + 2] : 0.f, s2);
            add(c3, csr.uw ? csr.uw[e + 3] : 0.f, s3);
        }
        for (; e < e_end; ++e) add(csr.ucol[e], csr.uw ? csr.uw[e] : 0.f, row_of(csr.ucol[e]));
        acc[0] += f0;
        acc[1] += f1;
        acc[2] += f2;
        acc[3] += f3;
    }
    if (!one_graph) {
        if (valid) flush();
        return;   // uniform across the block: every thread took this branch
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) red[threadIdx.y][threadIdx.x][c] = (double)acc[c];
    __syncthreads();
    if (threadIdx.y == 0 && valid) {
        const int g = csr.node_graph[chunk0];
        double* dst = agree + ((int64_t)g * row_stride + k) * R_pad + 4 * quad;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = 0.0;
#pragma unroll
            for (int y = 0; y < kScoreLanes; ++y) v += red[y][threadIdx.x][c];
            if (v != 0.0) atomicAdd(dst + c, v);
        }
    }
}

// E_r = sum_{i<j} w_ij cos(2 pi (theta_i - theta_j)) with FP32 terms, FP64 sum.
__global__ void __launch_bounds__(256) energy_kernel(CSRDev csr, const float* __restrict__ theta,
                                                     int R_pad, double* __restrict__ energy, int npt) {
    const int quads = R_pad >> 2;
    const int quad = blockIdx.x * blockDim.x + threadIdx.x;
    if (quad >= quads) return;
    const int first = blockIdx.y * npt;
    const int last = min(first + npt, csr.nodes);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int g_cur = -1;
    auto flush = [&]() {
        if (g_cur < 0) return;
        double* dst = energy + (int64_t)g_cur * R_pad + 4 * quad;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (acc[c] != 0.0) atomicAdd(dst + c, acc[c]);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = 0.0;
    };
    for (int node = first; node < last; ++node) {
        const int g = csr.node_graph[node];
        if (g != g_cur) {
            flush();
            g_cur = g;
        }
        const float4 ti = *reinterpret_cast<const float4*>(theta + (size_t)node * R_pad + 4 * quad);
        const int e_end = csr.rowp[node + 1];
        for (int e = csr.rowp[node]; e < e_end; ++e) {
            const uint32_t cw = csr.col[e];
            const uint32_t j = checked_node(csr, g, csr.w ? cw : (cw & ~kSignBit), (uint32_t)node);
            if ((int)j <= node) continue;
            const float w = csr.w ? csr.w[e] : ((cw & kSignBit) ? -1.0f : 1.0f);
            const float4 tj = *reinterpret_cast<const float4*>(theta + (size_t)j * R_pad + 4 * quad);
            acc[0] += (double)(w * cospif(2.0f * (ti.x - tj.x)));
            acc[1] += (double)(w * cospif(2.0f * (ti.y - tj.y)));
            acc[2] += (double)(w * cospif(2.0f * (ti.z - tj.z)));
            acc[3] += (double)(w * cospif(2.0f * (ti.w - tj.w)));
        }
    }
    flush();
}

// score[g][r] from the agreeing weight: q == 2 the cut wtot - agree, else agree.
__global__ void finalize_kernel(const GraphDev* __restrict__ graphs, int G, int q, int R, int R_pad,
                                const double* __restrict__ agree, int64_t row_stride, int64_t k,
                                double* __restrict__ score) {
    const int g = blockIdx.y;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || r >= R) return;
    const double a = agree[((int64_t)g * row_stride + k) * R_pad + r];
    score[(int64_t)g * R + r] = (q == 2) ? graphs[g].wtot - a : a;
}

// theta[node][R_pad] -> out[g][r][i] for spins (FP32 readout) and / or phases.
__global__ void gather_kernel(CSRDev csr, const float* __restrict__ theta, int R, int R_pad, int q,
                              int8_t* __restrict__ spins, float* __restrict__ th_out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)csr.nodes * R) return;
    // output index order: graph, replica, node
    // find the graph by scanning node offsets (G is small)
    int64_t rem = gid;
    int g = 0;
    for (; g < csr.G; ++g) {
        const int64_t span = (int64_t)csr.graphs[g].n * R;
        if (rem < span) break;
        rem -= span;
    }
    const int n = csr.graphs[g].n;
    const int r = (int)(rem / n);
    const int i = (int)(rem - (int64_t)r * n);
    const int node = csr.graphs[g].node_off + i;
    const float th = theta[(size_t)node * R_pad + r];
    if (spins) spins[gid] = (int8_t)spin_of(th, q);
    if (th_out) th_out[gid] = th;
}

// Nodes per thread of the edge passes: few enough that the grid holds about
// 2048 threads per SM (the passes are latency bound: one dependent gather per
// edge), at most 16 so that the FP64 atomics stay few when the grid is large.
int nodes_per_thread(const oim_run_s& r) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = v;
        else
            sms = 152;
    }
    const int64_t quads = r.R_pad / 4;
    const int64_t want = (int64_t)sms * 2048;
    const int64_t npt = (int64_t)r.p->nodes * quads / want;
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, npt));
}

}  // namespace

cudaError_t launch_score_at(const oim_run_s& r, const float* theta, int64_t k, const int32_t* d_t0,
                            int32_t t_add, cudaStream_t s);

cudaError_t launch_score(const oim_run_s& r, const float* theta, int64_t k, cudaStream_t s) {
    return launch_score_at(r, theta, k, nullptr, 0, s);
}

// The spins of every node-replica into d_spins (the first half of a score pass).
cudaError_t launch_spins(const oim_run_s& r, const float* theta, cudaStream_t s) {
    const int64_t quads_total = (int64_t)r.p->nodes * (r.R_pad / 4);
    spin_kernel<<<(unsigned)((quads_total + 255) / 256), 256, 0, s>>>(theta, quads_total, r.p->q, r.d_spins);
    return cudaGetLastError();
}

// The agreeing weights of every replica from d_spins into readout slot k (the second
// half); with d_t0 the slot is (*d_t0 + t_add) / readout_every - 1, read on the device.
cudaError_t launch_score_pass(const oim_run_s& r, int64_t k, const int32_t* d_t0, int32_t t_add, cudaStream_t s) {
    const int quads = r.R_pad / 4;
    const int npt = nodes_per_thread(r);
    const int chunk = kScoreLanes * npt;
    dim3 block(kScoreQuads, kScoreLanes);
    int max_deg = 0;
    for (const GraphDev& gd : r.p->graphs) max_deg = std::max(max_deg, gd.max_deg);
    const bool f32_sums = r.p->unit_weights && (int64_t)npt * max_deg < (int64_t)1 << 24;
    // the node ranges whose graphs are not scored on the tensor cores (all nodes by default)
    const int2 all = make_int2(0, (int)r.p->nodes);
    const int2* rg = r.score_split ? r.score_ranges.data() : &all;
    const size_t nr = r.score_split ? r.score_ranges.size() : 1;
    for (size_t q = 0; q < nr; ++q) {
        if (rg[q].y <= rg[q].x) continue;
        dim3 grid((quads + kScoreQuads - 1) / kScoreQuads, (unsigned)((rg[q].y - rg[q].x + chunk - 1) / chunk));
        const auto fn = f32_sums ? score_kernel<true> : score_kernel<false>;
        fn<<<grid, block, 0, s>>>(r.p->csr(), r.d_spins, r.R_pad, r.d_trace, r.readouts_cap, k, npt, d_t0, t_add,
                                  (int32_t)std::max<int64_t>(1, r.readout_every), rg[q].x, rg[q].y);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_score_at(const oim_run_s& r, const float* theta, int64_t k, const int32_t* d_t0,
                            int32_t t_add, cudaStream_t s) {
    cudaError_t e = launch_spins(r, theta, s);
    return e == cudaSuccess ? launch_score_pass(r, k, d_t0, t_add, s) : e;
}

cudaError_t launch_finalize(const oim_run_s& r, int64_t k, double* score, cudaStream_t s) {
    dim3 block(128);
    dim3 grid((r.R + 127) / 128, r.p->G);
    finalize_kernel<<<grid, block, 0, s>>>(r.p->d_graphs, r.p->G, r.p->q, r.R, r.R_pad, r.d_trace,
                                           r.readouts_cap, k, score);
    return cudaGetLastError();
}

cudaError_t launch_energy_of(const oim_run_s& r, const float* theta, double* energy, cudaStream_t s) {
    const int quads = r.R_pad / 4;
    dim3 block(min(256, ((quads + 31) / 32) * 32));
    const int npt = nodes_per_thread(r);
    dim3 grid((quads + block.x - 1) / block.x, (unsigned)((r.p->nodes + npt - 1) / npt));
    energy_kernel<<<grid, block, 0, s>>>(r.p->csr(), theta, r.R_pad, energy, npt);
    return cudaGetLastError();
}

cudaError_t launch_gather(const oim_run_s& r, const float* theta, int8_t* spins, float* th_out,
                          cudaStream_t s) {
    const int64_t total = r.p->nodes * r.R;
    const int threads = 256;
    gather_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(
        r.p->csr(), theta, r.R, r.R_pad, r.p->q, spins, th_out);
    return cudaGetLastError();
}

}  // namespace oim

// step_stream.cu -- the plain FP32 CSR form: one launch per Euler-Maruyama step,
// all state in device memory.
//
// Layout: theta[node][R_pad] (FP32) and cs[node][R_pad] = (cos 2 pi theta,
// sin 2 pi theta) as float2, replicas contiguous.  One thread owns one node and
// a quad of four consecutive replicas, so every neighbour gather is two 16-byte
// loads that a warp turns into fully used 128-byte lines, and one Philox block
// feeds the four noise draws of the quad.
//
// Per step and node (Eq. 5 / Algorithm 1, synchronous update from the old phases,
// written to the other buffer as in Sec. III-B):
//   (A, B)   = sum_j w_ij (cos 2 pi theta_j, sin 2 pi theta_j)
//   D_i      = sin(2 pi theta_i) A - cos(2 pi theta_i) B = sum_j w_ij sin 2 pi (theta_i - theta_j)
//   theta_i' = wrap(theta_i + dt (K D_i - Ks sin 2 pi q theta_i) + Kn sqrt(dt) xi)
//   cs_i'    = (cos 2 pi theta_i', sin 2 pi theta_i')
#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {

namespace {

__global__ void __launch_bounds__(256) init_stream_kernel(CSRDev csr, StepParams P,
                                                          float* __restrict__ theta,
                                                          float2* __restrict__ cs) {
    const int pairs = P.R_pad >> 1;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)csr.nodes * pairs) return;
    const int node = (int)(gid / pairs);
    const int r = 2 * (int)(gid - (int64_t)node * pairs);
    const int g = csr.node_graph[node];
    const int i = node - csr.graphs[g].node_off;
    const float2 th = init_pair(P.seed, (uint32_t)g, (uint32_t)i, (uint32_t)r);
    const size_t at = (size_t)node * P.R_pad + r;
    *reinterpret_cast<float2*>(theta + at) = th;
    float s0, c0, s1, c1;
    sincospif(2.0f * th.x, &s0, &c0);
    sincospif(2.0f * th.y, &s1, &c1);
    *reinterpret_cast<float4*>(cs + at) = make_float4(c0, s0, c1, s1);
}

template <bool kUnit>
__global__ void __launch_bounds__(256) step_stream_kernel(CSRDev csr, StepParams P,
                                                          const float* __restrict__ th_in,
                                                          const float2* __restrict__ cs_in,
                                                          float* __restrict__ th_out,
                                                          float2* __restrict__ cs_out,
                                                          int64_t t_fixed,
                                                          const int32_t* __restrict__ d_t0,
                                                          int32_t t_add) {
    const int quads = P.R_pad >> 2;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)csr.nodes * quads) return;
    const int node = (int)(gid / quads);
    const int quad = (int)(gid - (int64_t)node * quads);
    const int g = csr.node_graph[node];
    const int i = node - csr.graphs[g].node_off;
    const int64_t t = d_t0 ? (int64_t)(*d_t0) + t_add : t_fixed;
    const size_t sidx = (size_t)g * P.steps + t;
    const float K = __ldg(P.K + sidx), Ks = __ldg(P.Ks + sidx), Kn = __ldg(P.Kn + sidx);

    const size_t at = (size_t)node * P.R_pad + 4 * quad;
    const float4 th = *reinterpret_cast<const float4*>(th_in + at);
    const float4 o01 = *reinterpret_cast<const float4*>(cs_in + at);
    const float4 o23 = *reinterpret_cast<const float4*>(cs_in + at + 2);

    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    const int e_end = __ldg(csr.rowp + node + 1);
    for (int e = __ldg(csr.rowp + node); e < e_end; ++e) {
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
        const float4* nb = reinterpret_cast<const float4*>(cs_in + (size_t)j * P.R_pad + 4 * quad);
        const float4 v01 = __ldg(nb);
        const float4 v23 = __ldg(nb + 1);
        const float2 ww = make_float2(w, w);
        a0 = ffma2(make_float2(v01.x, v01.y), ww, a0);
        a1 = ffma2(make_float2(v01.z, v01.w), ww, a1);
        a2 = ffma2(make_float2(v23.x, v23.y), ww, a2);
        a3 = ffma2(make_float2(v23.z, v23.w), ww, a3);
    }

    const uint4 x = draw_block(P.seed, (uint32_t)g, kStreamNoise, (uint32_t)i, (uint32_t)t,
                               (uint32_t)quad);
    const float2 z01 = box_muller(x.x, x.y);
    const float2 z23 = box_muller(x.z, x.w);
    const float kick = Kn * P.sqrt_dt;
    const float dtK = P.dt * K, dtKs = P.dt * Ks;

    auto update = [&](float th0, float c, float s, float2 a, float z) {
        const float coup = s * a.x - c * a.y;
        const float shil = sin_q(P.q, c, s);
        return wrap01(th0 + (dtK * coup - dtKs * shil) + kick * z);
    };
    float4 tn;
    tn.x = update(th.x, o01.x, o01.y, a0, z01.x);
    tn.y = update(th.y, o01.z, o01.w, a1, z01.y);
    tn.z = update(th.z, o23.x, o23.y, a2, z23.x);
    tn.w = update(th.w, o23.z, o23.w, a3, z23.y);
    *reinterpret_cast<float4*>(th_out + at) = tn;
    float4 n01, n23;
    sincospif(2.0f * tn.x, &n01.y, &n01.x);
    sincospif(2.0f * tn.y, &n01.w, &n01.z);
    sincospif(2.0f * tn.z, &n23.y, &n23.x);
    sincospif(2.0f * tn.w, &n23.w, &n23.z);
    *reinterpret_cast<float4*>(cs_out + at) = n01;
    *reinterpret_cast<float4*>(cs_out + at + 2) = n23;
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
        const uint32_t j = csr.w ? cw : (cw & ~kSignBit);
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
    P.q = r.p->q;
    P.R = r.R;
    P.R_pad = r.R_pad;
    return P;
}

StepParams make_params(const oim_run_s& r) { return params_of(r); }

cudaError_t launch_init_stream(const oim_run_s& r, cudaStream_t s) {
    const StepParams P = params_of(r);
    const int64_t total = r.p->nodes * (r.R_pad / 2);
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    init_stream_kernel<<<(unsigned)blocks, threads, 0, s>>>(
        r.p->csr(), P, r.d_theta[0], reinterpret_cast<float2*>(r.d_cs[0]));
    return cudaGetLastError();
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

// One step t of the stream form between explicit buffers.
cudaError_t launch_step_stream_buffers(const oim_run_s& r, int64_t t, const float* th_in,
                                       const float2* cs_in, float* th_out, float2* cs_out,
                                       cudaStream_t s) {
    const StepParams P = params_of(r);
    const int64_t total = r.p->nodes * (r.R_pad / 4);
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    if (r.p->unit_weights)
        step_stream_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, nullptr, 0);
    else
        step_stream_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_step_stream(const oim_run_s& r, int64_t t, const int32_t* d_t0, cudaStream_t s) {
    // with d_t0 the step is *d_t0 + t (graph replay); otherwise t itself.
    const StepParams P = params_of(r);
    const int64_t total = r.p->nodes * (r.R_pad / 4);
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    const int in = (int)(t & 1);   // buffer parity follows the step index
    const int out = in ^ 1;
    const float* th_in = r.d_theta[in];
    const float2* cs_in = reinterpret_cast<const float2*>(r.d_cs[in]);
    float* th_out = r.d_theta[out];
    float2* cs_out = reinterpret_cast<float2*>(r.d_cs[out]);
    if (r.p->unit_weights)
        step_stream_kernel<true><<<(unsigned)blocks, threads, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, d_t0, (int32_t)t);
    else
        step_stream_kernel<false><<<(unsigned)blocks, threads, 0, s>>>(
            r.p->csr(), P, th_in, cs_in, th_out, cs_out, t, d_t0, (int32_t)t);
    return cudaGetLastError();
}

}  // namespace oim

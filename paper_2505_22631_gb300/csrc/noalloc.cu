// noalloc.cu -- oim_score_phases_noalloc: the score pass of oim_readout for
// caller-supplied phases, with its accumulators in a fixed, file-scope device
// array instead of memory obtained from cudaMalloc.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "oim_checks.cuh"
#include "oim_device.cuh"
#include "oim_internal.h"

namespace oim {
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
}  // namespace oim

using namespace oim;

namespace {

// Scratch of the no-allocation entry point: agreeing weight per (graph, replica).
static __device__ __align__(256) double g_noalloc_accum[OIM_NOALLOC_MAX_ACCUM];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_accum_ptr[kMaxDevices] = {nullptr};

constexpr int kNodesPerThread = 16;
constexpr unsigned kMaxGridY = 65535;   // the grid's y extent; chunks beyond it are strided

// sum_{i<j} w_ij [spin_i == spin_j] per (graph, replica) into accum[g * ld + r].
// Thread = (replica quad, chunks of kNodesPerThread nodes: blockIdx.y, then every
// gridDim.y-th chunk after it, so that any node count fits the grid).
__global__ void __launch_bounds__(256) noalloc_agree_kernel(CSRDev csr, const float* __restrict__ theta,
                                                            int ld, int q, double* __restrict__ accum) {
    const int quads = ld >> 2;
    const int quad = blockIdx.x * blockDim.x + threadIdx.x;
    if (quad >= quads) return;
    const int chunks = (csr.nodes + kNodesPerThread - 1) / kNodesPerThread;
    for (int chunk = blockIdx.y; chunk < chunks; chunk += gridDim.y) {
    const int first = chunk * kNodesPerThread;
    const int last = min(first + kNodesPerThread, csr.nodes);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int g_cur = -1;
    auto flush = [&]() {
        if (g_cur < 0) return;
        double* dst = accum + (int64_t)g_cur * ld + 4 * quad;
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
        const float4 ti = *reinterpret_cast<const float4*>(theta + (size_t)node * ld + 4 * quad);
        const int s0 = spin_of(ti.x, q), s1 = spin_of(ti.y, q), s2 = spin_of(ti.z, q),
                  s3 = spin_of(ti.w, q);
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
        for (int e = csr.rowp[node]; e < csr.rowp[node + 1]; ++e) {
            const uint32_t cw = csr.col[e];
            const uint32_t j = checked_node_of_row(csr, node, csr.w ? cw : (cw & ~kSignBit));
            if ((int)j <= node) continue;
            const float w = csr.w ? csr.w[e] : ((cw & kSignBit) ? -1.0f : 1.0f);
            const float4 tj = *reinterpret_cast<const float4*>(theta + (size_t)j * ld + 4 * quad);
            f0 += (s0 == spin_of(tj.x, q)) ? w : 0.f;
            f1 += (s1 == spin_of(tj.y, q)) ? w : 0.f;
            f2 += (s2 == spin_of(tj.z, q)) ? w : 0.f;
            f3 += (s3 == spin_of(tj.w, q)) ? w : 0.f;
        }
        acc[0] += f0;
        acc[1] += f1;
        acc[2] += f2;
        acc[3] += f3;
    }
    flush();
    }
}

// score[g][r] = wtot_g - agree (q == 2) or agree (q >= 3).
__global__ void noalloc_finalize_kernel(const GraphDev* __restrict__ graphs, int G, int q, int R,
                                        int ld, const double* __restrict__ accum,
                                        double* __restrict__ score) {
    const int g = blockIdx.y;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || r >= R) return;
    const double a = accum[(int64_t)g * ld + r];
    score[(int64_t)g * R + r] = (q == 2) ? graphs[g].wtot - a : a;
}

bool device_pointer(const void* ptr) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return fail(OIM_EUNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_accum_ptr[device]) {
        double* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_accum);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_accum_ptr[device] = ptr;
    }
    *out = g_accum_ptr[device];
    return OIM_OK;
}

}  // namespace

extern "C" int oim_score_phases_noalloc(oim_problem_t p, const float* theta, int32_t replicas,
                                        int32_t ld, double* score, void* stream) {
    if (!p || !theta || !score) return fail(OIM_EINVAL, "NULL argument");
    if (replicas < 1 || ld < replicas || ld % 4 != 0)
        return fail(OIM_EINVAL, "need 1 <= replicas <= ld and ld a multiple of 4");
    const int64_t need = (int64_t)p->G * ld;
    if (need > OIM_NOALLOC_MAX_ACCUM)
        return fail(OIM_EINVAL, "graphs * ld = " + std::to_string(need) +
                                    " exceeds the no-allocation scratch of " +
                                    std::to_string(OIM_NOALLOC_MAX_ACCUM) + " doubles");
    // theta is read in 16-byte groups of four replicas and score written as doubles
    if (reinterpret_cast<uintptr_t>(theta) % 16 != 0)
        return fail(OIM_EINVAL, "theta must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(score) % sizeof(double) != 0)
        return fail(OIM_EINVAL, "score must be 8-byte aligned");
    if (!p->uploaded) return fail(OIM_ESTATE, "the problem's graph is not on the device yet");
    DeviceScope scope;   // the caller's current device is restored on return
    {
        cudaError_t e = scope.enter(p->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    }
    if (!device_pointer(theta) || !device_pointer(score))
        return fail(OIM_EINVAL, "theta and score must be device memory");
    double* accum = nullptr;
    int rc = scratch_address(p->device, &accum);
    if (rc != OIM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(accum, 0, (size_t)need * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "clear no-allocation scratch");
    const int quads = ld / 4;
    dim3 block(std::min(256, ((quads + 31) / 32) * 32));
    const int64_t chunks = (p->nodes + kNodesPerThread - 1) / kNodesPerThread;
    dim3 grid((quads + block.x - 1) / block.x, (unsigned)std::min<int64_t>(chunks, kMaxGridY));
    noalloc_agree_kernel<<<grid, block, 0, s>>>(p->csr(), theta, ld, p->q, accum);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation score launch");
    dim3 fblock(128);
    dim3 fgrid((replicas + 127) / 128, p->G);
    noalloc_finalize_kernel<<<fgrid, fblock, 0, s>>>(p->d_graphs, p->G, p->q, replicas, ld, accum, score);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation finalize launch");
    return OIM_OK;
}

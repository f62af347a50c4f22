// gemm_tc.cu -- tensor-core (tcgen05) building blocks of the dense coupling form:
// TMA tensor maps and a self-test GEMM that exercises the exact operand layouts,
// descriptors and TMEM read-back the fused step kernel uses.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]     (A: M x K, B: N x K, both bf16 row-major,
//                                          i.e. K-major operands; D fp32)
// One CTA per 128 x BN output tile; thread 0 streams 64-wide K blocks through a
// ring of shared-memory stages with TMA and issues tcgen05.mma (K = 16 each) into
// a TMEM accumulator; the four warps then read their 32 TMEM lanes back.
#include <mutex>
#include <string>

#include "oim_internal.h"
#include "tc_common.cuh"

namespace oim {

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

constexpr int kBM = 128;             // rows of a tile (TMEM lanes)
constexpr int kBK = 64;              // K block: 64 bf16 = one 128-byte swizzle row
constexpr int kABytes = kBM * 128;   // A stage: 128 rows x 128 B

// With withhold >= 0 the producer skips the TMA load of K block `withhold`: the MMA
// thread's wait for it then runs out after `polls` polls and records the error, the
// loads already in flight are waited for (bounded), the TMEM is freed and the block
// returns -- the path every bounded wait of the pipeline takes when it gives up.
template <int BN, int S>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_test_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                        float* __restrict__ D, int M, int N, int K, int32_t* err, int withhold,
                        uint32_t polls) {
    using namespace tc;
    constexpr int kBBytes = BN * 128;
    constexpr uint32_t kCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + S * kABytes;
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_slot;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int KB = K / kBK;
    if (threadIdx.x == 0) {
        prefetch_map(&mA);
        prefetch_map(&mB);
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
        const uint32_t idesc = idesc_bf16_f32(kBM, BN);
        // K block loaded into each stage and not yet waited for (-1: none)
        int pending[S];
        auto load = [&](int kb) {
            const int s = kb % S;
            if (kb == withhold) return;   // withheld: nothing will arrive on full[s]
            mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
            tma_load_2d(sA + s * kABytes, &mA, kb * kBK, m0, &full[s]);
            tma_load_2d(sB + s * kBBytes, &mB, kb * kBK, n0, &full[s]);
            pending[s] = kb;
        };
        for (int s = 0; s < S; ++s) pending[s] = -1;
        for (int kb = 0; kb < KB && kb < S; ++kb) load(kb);
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            const int s = kb % S;
            if (!mbar_wait_polls(&full[s], (kb / S) & 1, err, kErrFullWait, polls)) {
                ok = false;
                break;
            }
            pending[s] = -1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                umma_bf16(tmem, sdesc_kmajor_sw128(a0 + 32 * k), sdesc_kmajor_sw128(b0 + 32 * k), idesc,
                          (kb | k) != 0);
            umma_commit(&empty[s]);
            if (kb + S < KB) {
                if (!mbar_wait_polls(&empty[s], (kb / S) & 1, err, kErrEmptyWait, polls)) {
                    ok = false;
                    break;
                }
                load(kb + S);
            }
        }
        // after a wait that gave up, let the loads still in flight land before the
        // shared memory they write is released
        for (int s = 0; s < S; ++s)
            if (pending[s] >= 0) mbar_wait_polls(&full[s], (pending[s] / S) & 1, err, kErrFullWait, polls);
        // completes when every MMA issued above has finished (also on the error path)
        umma_commit(&done);
    }
    __syncwarp();
    const bool have = mbar_wait_polls(&done, 0, err, kErrDoneWait, polls);
    tc_fence_after();
    if (have) {
        const int row = warp * 32 + lane;
        float* out = D + (size_t)(m0 + row) * N + n0;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[c + j] = __uint_as_float(v[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

}  // namespace

// 2-D bf16 tensor map over a rows x cols row-major matrix (pitch in bytes), boxes of
// 64 columns x box_rows rows, 128-byte swizzle.
int make_map_bf16(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint64_t pitch,
                  uint32_t box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(OIM_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {pitch};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(OIM_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return OIM_OK;
}

}  // namespace oim

using namespace oim;

namespace {

int tc_gemm_run(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K, int withhold,
                uint32_t polls) {
    if (!A || !B || !D) return fail(OIM_EINVAL, "NULL argument");
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64)
        return fail(OIM_EINVAL, "need M, N multiples of 128 and K a multiple of 64");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        return fail(OIM_EINVAL, "A and B must be 16-byte aligned");
    CUtensorMap mA, mB;
    int rc = make_map_bf16(&mA, A, (uint64_t)K, (uint64_t)M, (uint64_t)K * 2, 128);
    if (rc != OIM_OK) return rc;
    rc = make_map_bf16(&mB, B, (uint64_t)K, (uint64_t)N, (uint64_t)K * 2, 128);
    if (rc != OIM_OK) return rc;
    int32_t* d_err = nullptr;
    cudaError_t e = cudaMalloc(&d_err, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(err)");
    cudaMemset(d_err, 0, sizeof(int32_t));
    constexpr int S = 4;
    const size_t smem = (size_t)S * (128 * 128 + 128 * 128) + 1024;
    auto fn = tc_gemm_test_kernel<128, S>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        fn<<<dim3(N / 128, M / 128), 128, smem>>>(mA, mB, D, M, N, K, d_err, withhold, polls);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core self-test");
    if (err) return fail(OIM_ETIMEOUT, "tensor-core self-test: a pipeline wait gave up (" + std::to_string(err) + ")");
    return OIM_OK;
}

}  // namespace

extern "C" int oim_debug_tc_gemm(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K) {
    return tc_gemm_run(A, B, D, M, N, K, -1, tc::kWaitPolls);
}

extern "C" int oim_debug_tc_gemm_withhold(const void* A, const void* B, float* D, int32_t M, int32_t N,
                                          int32_t K, int32_t withhold_k_block, uint32_t wait_polls) {
    if (wait_polls < 1) return fail(OIM_EINVAL, "wait_polls must be >= 1");
    if (withhold_k_block < -1) return fail(OIM_EINVAL, "withhold_k_block must be >= -1");
    return tc_gemm_run(A, B, D, M, N, K, withhold_k_block, wait_polls);
}

// oim_device.cuh -- device helpers shared by the step, readout and adjoint kernels.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2), counter-based so that every
// draw is a pure function of (seed, graph, stream, node, step, replica) and no
// generator state is stored (the paper keeps per-thread cuRAND states, Sec. III-B).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace oim {

constexpr uint32_t kStreamInit = 0;
constexpr uint32_t kStreamNoise = 1;

// Ten Philox rounds: per round the pair products of c0 and c2 with the two
// multipliers are taken, their high halves are mixed with c1/c3 and the key,
// and the key advances by the two Weyl increments.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Two Philox blocks with the same key, advanced through one shared key schedule.
__device__ __forceinline__ void philox10_pair(uint4& a, uint4& b, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        // each 32 x 32-bit product whole (low and high words from one wide multiply)
        const uint64_t pa0 = (uint64_t)0xD2511F53u * a.x, pa1 = (uint64_t)0xCD9E8D57u * a.z;
        const uint64_t pb0 = (uint64_t)0xD2511F53u * b.x, pb1 = (uint64_t)0xCD9E8D57u * b.z;
        const uint32_t alo0 = (uint32_t)pa0, ahi0 = (uint32_t)(pa0 >> 32);
        const uint32_t alo1 = (uint32_t)pa1, ahi1 = (uint32_t)(pa1 >> 32);
        const uint32_t blo0 = (uint32_t)pb0, bhi0 = (uint32_t)(pb0 >> 32);
        const uint32_t blo1 = (uint32_t)pb1, bhi1 = (uint32_t)(pb1 >> 32);
        a = make_uint4(ahi1 ^ a.y ^ k0, alo1, ahi0 ^ a.w ^ k1, alo0);
        b = make_uint4(bhi1 ^ b.y ^ k0, blo1, bhi0 ^ b.w ^ k1, blo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Block of four words for (node i, step t, replica quad rq) of one graph/stream.
__device__ __forceinline__ uint4 draw_block(uint64_t seed, uint32_t graph, uint32_t stream,
                                            uint32_t i, uint32_t t, uint32_t rq) {
    return philox10(make_uint4(i, t, rq, (graph << 1) | stream), (uint32_t)seed,
                    (uint32_t)(seed >> 32));
}

// The blocks of replica quads rq and rq + 1 at (node i, step t) of one graph/stream.
__device__ __forceinline__ void draw_block_pair(uint64_t seed, uint32_t graph, uint32_t stream, uint32_t i,
                                                uint32_t t, uint32_t rq, uint4& a, uint4& b) {
    a = make_uint4(i, t, rq, (graph << 1) | stream);
    b = make_uint4(i, t, rq + 1, (graph << 1) | stream);
    philox10_pair(a, b, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ((x >> 9) + 1/2) * 2^-23: an odd multiple of 2^-24 in (0,1), exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) {
    return __fmaf_rn((float)(x >> 9), 0x1p-23f, 0x1p-24f);
}

// Box-Muller: rho = sqrt(-2 ln ua); (rho cos 2 pi ub, rho sin 2 pi ub).
__device__ __forceinline__ float2 box_muller(uint32_t xa, uint32_t xb) {
    const float ua = u01(xa);
    const float ub = u01(xb);
    const float rho = sqrtf(-2.0f * logf(ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);
    return make_float2(rho * c, rho * s);
}

// Hardware square-root approximation (PTX sqrt.approx.f32).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2 pi u mapped to [-pi, pi): u - 1 is exact for u in [1/2, 1).
__device__ __forceinline__ float turn_to_rad(float u) {
    return (u >= 0.5f ? u - 1.0f : u) * 6.28318530717958647f;
}

// Box-Muller with the hardware approximations of log2, sqrt, sin and cos
// (special function unit).  Same draws as box_muller to about 1e-6 absolute;
// used where the (cos, sin) cache is stored in 16 bits (rounding 2^-12).
__device__ __forceinline__ float2 box_muller_fast(uint32_t xa, uint32_t xb) {
    const float ua = u01(xa);
    const float ub = u01(xb);
    const float rho = sqrt_approx(-1.38629436111989061f * __log2f(ua));   // -2 ln 2 log2(ua)
    float s, c;
    __sincosf(turn_to_rad(ub), &s, &c);
    return make_float2(rho * c, rho * s);
}

// (cos 2 pi theta, sin 2 pi theta) for theta in [0,1) with the hardware sin / cos.
__device__ __forceinline__ float2 cos_sin_2pi_fast(float th) {
    float s, c;
    __sincosf(turn_to_rad(th), &s, &c);
    return make_float2(c, s);
}

// (cos, sin) of 2 pi (th + 1/2) = -(cos, sin)(2 pi th) for th in [0,1) with the
// hardware sin / cos: the argument 2 pi th - pi lies in [-pi, pi) and takes one FMA.
// Kernels that keep half-turn pairs for the own phase and the neighbours alike get
// the coupling sum_j w_ij sin 2 pi (theta_i - theta_j) unchanged (it depends on phase
// differences only) and fold the other signs into scalars.
__device__ __forceinline__ float2 cos_sin_half_turn_fast(float th) {
    float s, c;
    __sincosf(__fmaf_rn(th, 6.28318530717958647f, -3.14159265358979324f), &s, &c);
    return make_float2(c, s);
}

// Box-Muller like box_muller_fast with the angle 2 pi ub - pi: returns the negated
// pair of normals, -(rho cos 2 pi ub, rho sin 2 pi ub).
__device__ __forceinline__ float2 box_muller_half_turn_fast(uint32_t xa, uint32_t xb) {
    const float ua = u01(xa);
    const float ub = u01(xb);
    const float rho = sqrt_approx(-1.38629436111989061f * __log2f(ua));   // -2 ln 2 log2(ua)
    const float2 cs = cos_sin_half_turn_fast(ub);
    return make_float2(rho * cs.x, rho * cs.y);
}

// Normals for the replica pair (r, r+1), r even: lanes (r&3, r&3 + 1).
__device__ __forceinline__ float2 noise_pair(uint64_t seed, uint32_t graph, uint32_t i,
                                             uint32_t t, uint32_t r) {
    const uint4 x = draw_block(seed, graph, kStreamNoise, i, t, r >> 2);
    return (r & 2) ? box_muller(x.z, x.w) : box_muller(x.x, x.y);
}

// Initial phases of the replica pair (r, r+1), r even.
__device__ __forceinline__ float2 init_pair(uint64_t seed, uint32_t graph, uint32_t i,
                                            uint32_t r) {
    const uint4 x = draw_block(seed, graph, kStreamInit, i, 0, r >> 2);
    return (r & 2) ? make_float2(u01(x.z), u01(x.w)) : make_float2(u01(x.x), u01(x.y));
}

// theta - floor(theta) in [0,1); a tiny negative theta rounds up to 1.0f and maps to 0.
__device__ __forceinline__ float wrap01(float x) {
    float y = x - floorf(x);
    return (y >= 1.0f) ? 0.0f : y;
}

// sin(2 pi q theta) from (c, s) = (cos 2 pi theta, sin 2 pi theta).
__device__ __forceinline__ float sin_q(int q, float c, float s) {
    if (q == 2) return 2.0f * s * c;
    if (q == 3) return s * __fmaf_rn(-4.0f * s, s, 3.0f);
    // sin((m+1)x) = 2 cos(x) sin(mx) - sin((m-1)x)
    float prev = 0.0f, cur = s;
    for (int m = 1; m < q; ++m) {
        const float nxt = __fmaf_rn(2.0f * c, cur, -prev);
        prev = cur;
        cur = nxt;
    }
    return cur;
}

// Nearest stable phase k/q: floor(q*theta + 1/2) mod q, each operation rounded
// to FP32 separately (no contraction) so that host and device decide alike.
__device__ __forceinline__ int spin_of(float theta, int q) {
    const float a = __fmul_rn((float)q, theta);
    const float b = __fadd_rn(a, 0.5f);
    const int k = (int)floorf(b);
    return (k >= q) ? k - q : k;
}

// acc += the two 16-bit halves of h2 (FP16 or BF16), each converted exactly and
// added with one FP32 rounding: the mixed-precision add of the sm_100 family.
__device__ __forceinline__ void add_f16x2(float2& acc, uint32_t h2) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "add.rn.f32.f16 %0, l, %0;\n\tadd.rn.f32.f16 %1, h, %1;\n\t}"
        : "+f"(acc.x), "+f"(acc.y) : "r"(h2));
}
__device__ __forceinline__ void add_bf16x2(float2& acc, uint32_t h2) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "add.rn.f32.bf16 %0, l, %0;\n\tadd.rn.f32.bf16 %1, h, %1;\n\t}"
        : "+f"(acc.x), "+f"(acc.y) : "r"(h2));
}

// acc = (the two 16-bit halves of h2) - acc, each with one FP32 rounding: the mixed
// subtract that turns an accumulator into the negated sum of the -1 entries that follow
// (-(acc - x) rounded to nearest equals x - acc rounded to nearest).
__device__ __forceinline__ void rsub_f16x2(float2& acc, uint32_t h2) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "sub.rn.f32.f16 %0, l, %0;\n\tsub.rn.f32.f16 %1, h, %1;\n\t}"
        : "+f"(acc.x), "+f"(acc.y) : "r"(h2));
}
__device__ __forceinline__ void rsub_bf16x2(float2& acc, uint32_t h2) {
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "sub.rn.f32.bf16 %0, l, %0;\n\tsub.rn.f32.bf16 %1, h, %1;\n\t}"
        : "+f"(acc.x), "+f"(acc.y) : "r"(h2));
}

// 32-byte global loads and stores (the sm_100 family's 256-bit vector accesses); the
// address must be 32-byte aligned.  ld256_nc reads data that no thread writes during
// the kernel (read-only path); ld256 reads data the kernel itself writes afterwards.
__device__ __forceinline__ void ld256_nc(const void* p, uint32_t (&r)[8]) {
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}
__device__ __forceinline__ void ld256_cg(const void* p, uint32_t (&r)[8]) {
    asm volatile("ld.global.cg.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void ld256(const void* p, uint32_t (&r)[8]) {
    asm("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "l"(p));
}
__device__ __forceinline__ void st256(void* p, const uint32_t (&r)[8]) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(r[0]), "r"(r[1]),
                 "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
}

}  // namespace oim

// Device helpers shared by the QC decoder kernels: the check-node transform
// phi, lane-word packing of V frames, and the per-package flag layout.
#pragma once

#include "ldpc_internal.cuh"

#include <mutex>
#include <unordered_map>

namespace ldpc {

constexpr int kWarps = 8;  // warps per block in the node kernels: 8 consecutive rows / variables

// ---------------------------------------------------------------------------
// phi(x) = -ln tanh(x/2) = ln((1 + e^-x)/(1 - e^-x)), x >= 0; phi(0) = +inf,
// phi(+inf) = 0, and phi is its own inverse, so eq. (bphs) becomes
// alpha = sign * phi(sum of phi(|beta|) over the other edges).
//
// Errors of a few ulp here grow by two orders of magnitude over 30 iterations
// on frames that do not converge, and phi is evaluated twice per edge, so it
// has to be both accurate and cheap.  Two regimes, both evaluated and selected
// (no divergence):
//  x >= 1:  phi = 2 atanh(t), t = e^-x <= 0.368, written 2 t S(t^2) with
//           S(v) = atanh(sqrt v)/sqrt v; t from the SFU exp2 with the
//           rounding error of x*log2(e) carried to first order.
//  x <  1:  phi = -ln(x/2) + G(x^2/4), G(u) = -ln(tanh(sqrt u)/sqrt u); the
//           log from the SFU log2 (its argument stays below 1/2, where the
//           approximation has a relative error bound), G a polynomial.
// S - 1 and G are degree-4 polynomials fitted here (weighted least squares
// converging to the minimax fit) to 1.3e-8 relative / 3.8e-9 absolute on
// their intervals; the remaining error is that of the SFU approximations.
// phi_ref keeps CUDA's expm1f/log1pf form (about 2-3 ulp, several times
// slower) for verification through ldpc_phi_eval.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float phi_ref(float x) {
    const float e = expm1f(x);
    return log1pf(2.0f * __frcp_rn(e));
}

__device__ __forceinline__ float ex2_approx(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float lg2_approx(float a) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// x >= 1 and finite (CLAMP: x may also be +inf)
template <bool CLAMP = true>
__device__ __forceinline__ float phi_hi(float x) {
    if (CLAMP) x = fminf(x, 100.0f);  // e^-100 flushes to 0; keeps inf - inf out of the error term
    const float L2E = 1.44269502f, L2E_LO = 1.92596299e-8f, LN2 = 0.693147182f;
    const float a = -x * L2E;
    float alo = fmaf(-x, L2E, -a);
    alo = fmaf(-x, L2E_LO, alo);
    const float t0 = ex2_approx(a);
    const float t = fmaf(t0, alo * LN2, t0);
    const float v = t * t;
    const float w = 2.0f * t;
    const float sv = v * fmaf(fmaf(fmaf(0.147845685f, v, 0.138392285f), v, 0.200207084f), v, 0.333330393f);
    return fmaf(w, sv, w);
}

__device__ __forceinline__ float phi_lo(float x) {  // 0 <= x < 1
    const float LN2 = 0.693147182f;
    const float y = 0.5f * x;
    const float u = y * y;
    const float G = u * fmaf(fmaf(fmaf(-0.00555368373f, u, 0.0216362253f), u, -0.0777590200f), u, 0.333332866f);
    return fmaf(lg2_approx(y), -LN2, G);
}

// Both regimes evaluated and selected: no branch.  (Voting per warp to
// evaluate one regime only costs more than it saves once the frames of a
// warp are at different iterations, as in the continuous simulation.)
__device__ __forceinline__ float phi_f(float x) {
    const float hi = phi_hi(x), lo = phi_lo(x);
    return x < 1.0f ? lo : hi;
}
// the same for finite x (no clamp)
__device__ __forceinline__ float phi_fin(float x) {
    const float hi = phi_hi<false>(x), lo = phi_lo(x);
    return x < 1.0f ? lo : hi;
}
// ---------------------------------------------------------------------------
// Packed pairs: the sm_100-family FP32x2 instructions (add/mul/fma .rn.f32x2) do two
// IEEE binary32 operations, each rounded to nearest-even, per issue slot.  phi2 /
// phi_fin2 run phi_f / phi_fin on two arguments with exactly the scalar versions'
// operations (so the results are bit-identical), halving the issue cost of the
// polynomial and error-term arithmetic; ex2/lg2 and the min/select stay scalar.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2split(f32x2 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 f2mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 f2c(float c) { return f2(c, c); }

// phi_hi of two arguments (already clamped when CLAMP is wanted), as pairs
__device__ __forceinline__ f32x2 phi_hi2(f32x2 x) {
    const float L2E = 1.44269502f, L2E_LO = 1.92596299e-8f, LN2 = 0.693147182f;
    const f32x2 a = f2mul(x, f2c(-L2E));         // -x * L2E
    const f32x2 na = f2mul(x, f2c(L2E));         // -a, exactly
    f32x2 alo = f2fma(x, f2c(-L2E), na);         // fmaf(-x, L2E, -a)
    alo = f2fma(x, f2c(-L2E_LO), alo);           // fmaf(-x, L2E_LO, alo)
    float a0, a1;
    f2split(a, a0, a1);
    const f32x2 t0 = f2(ex2_approx(a0), ex2_approx(a1));
    const f32x2 t = f2fma(t0, f2mul(alo, f2c(LN2)), t0);
    const f32x2 v = f2mul(t, t);
    const f32x2 w = f2mul(f2c(2.0f), t);
    f32x2 P = f2fma(f2c(0.147845685f), v, f2c(0.138392285f));
    P = f2fma(P, v, f2c(0.200207084f));
    P = f2fma(P, v, f2c(0.333330393f));
    const f32x2 sv = f2mul(v, P);
    return f2fma(w, sv, w);
}
__device__ __forceinline__ f32x2 phi_lo2(f32x2 x) {
    const float LN2 = 0.693147182f;
    const f32x2 y = f2mul(f2c(0.5f), x);
    const f32x2 u = f2mul(y, y);
    f32x2 G = f2fma(f2c(-0.00555368373f), u, f2c(0.0216362253f));
    G = f2fma(G, u, f2c(-0.0777590200f));
    G = f2fma(G, u, f2c(0.333332866f));
    G = f2mul(u, G);
    float y0, y1;
    f2split(y, y0, y1);
    return f2fma(f2(lg2_approx(y0), lg2_approx(y1)), f2c(-LN2), G);
}
// phi_f of (x0, x1)
__device__ __forceinline__ void phi2(float x0, float x1, float &y0, float &y1) {
    float h0, h1, l0, l1;
    f2split(phi_hi2(f2(fminf(x0, 100.0f), fminf(x1, 100.0f))), h0, h1);
    f2split(phi_lo2(f2(x0, x1)), l0, l1);
    y0 = x0 < 1.0f ? l0 : h0;
    y1 = x1 < 1.0f ? l1 : h1;
}
// phi_fin of (x0, x1) (finite arguments, no clamp)
__device__ __forceinline__ void phi_fin2(float x0, float x1, float &y0, float &y1) {
    const f32x2 x = f2(x0, x1);
    float h0, h1, l0, l1;
    f2split(phi_hi2(x), h0, h1);
    f2split(phi_lo2(x), l0, l1);
    y0 = x0 < 1.0f ? l0 : h0;
    y1 = x1 < 1.0f ? l1 : h1;
}

// Transformed message storage (the variable pass stores what the check pass sums):
// FP32 keeps sign(beta) * phi(|beta|); FP16 keeps it scaled by 2^12, so that the
// normal range of halves covers phi of |beta| in [2.3e-7, 18.7] -- a larger phi
// (|beta| ~ 0) overflows to inf, whose check-pass sum gives the other edges
// alpha = phi(inf) = 0, the limit of an erased input; a smaller one (|beta| > 18.7)
// keeps fewer digits and flushes to 0 past |beta| ~ 25.6, the limit of a certain input.
template <int V>
struct XfScale {
    static constexpr float store = 1.0f, load = 1.0f;
};
template <>
struct XfScale<2> {
    static constexpr float store = 4096.0f, load = 1.0f / 4096.0f;
};

// |y| with the sign bit of s
__device__ __forceinline__ float with_sign_of(float y, float s) {
    return __uint_as_float(__float_as_uint(y) | (__float_as_uint(s) & 0x80000000u));
}

__device__ __forceinline__ float clipf(float x, float c) { return fminf(fmaxf(x, -c), c); }

// lane word <-> V floats
template <int V> struct Lane;
template <> struct Lane<1> {
    static __device__ __forceinline__ void unpack(uint32_t w, float *x) { x[0] = __uint_as_float(w); }
    static __device__ __forceinline__ uint32_t pack(const float *x) { return __float_as_uint(x[0]); }
};
template <> struct Lane<2> {
    static __device__ __forceinline__ void unpack(uint32_t w, float *x) {
        __half2 h = *reinterpret_cast<__half2 *>(&w);
        float2 f = __half22float2(h);
        x[0] = f.x;
        x[1] = f.y;
    }
    static __device__ __forceinline__ uint32_t pack(const float *x) {
        __half2 h = __floats2half2_rn(x[0], x[1]);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

// flags of one package (V words per field; bit = lane)
struct PkgFlags {
    uint32_t *base;
    int V;
    __device__ uint32_t *done() const { return base; }
    __device__ uint32_t *unsat(int par) const { return base + (1 + par) * V; }
    __device__ uint32_t *valid() const { return base + 3 * V; }
    __device__ uint32_t *fin() const { return base + 4 * V; }
};


// ---------------------------------------------------------------------------
// Channel: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t *o) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
    o[3] = c3;
}

// ---------------------------------------------------------------------------
// The channel generator in binary32, defined operation by operation so that every
// implementation of it gives the same bits (the CPU reference implements the same
// definition).  Each step is one IEEE binary32 operation rounded to nearest-even,
// written with the _rn intrinsics so that the compiler cannot fuse or reorder it.
//
// Uniform of a Philox word w: u = v 2^-24 with v = 2 floor(w / 2^9) + 1 (odd, exact).
// ln u: u = m 2^e, m in [sqrt(1/2), sqrt(2)) from the bit pattern (threshold 0x3fb504f3),
//   f = m - 1 (exact), ln(1 + f) = f + f^2 (-1/2 + f R(f)) with R a degree-7 minimax
//   polynomial, ln u = e LN2_HI + (e LN2_LO + ln(1 + f)) (Cody-Waite split of ln 2;
//   LN2_HI has 15 significant bits, so e LN2_HI is exact).
// sin/cos of 2 pi u: the nearest quarter turn j = floor((v + 2^21) / 2^22) and
//   r = (v - j 2^22) 2^-24 in [-1/8, 1/8] (exact integer steps), sin(2 pi r) = r S(r^2),
//   cos(2 pi r) = 1 + r^2 C(r^2) with degree-4 minimax polynomials; the quadrant j mod 4
//   swaps and negates them.
// Coefficients: binary32 minimax fits (Lawson's algorithm) made for this generator.
// Accuracy (all 2^23 inputs): ln 0.87 ulp, sin and cos 1.6 ulp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float chan_ln(float u) {
    const uint32_t b = __float_as_uint(u);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    if (mb > 0x3fb504f3u) {
        mb -= 0x00800000u;
        e += 1;
    }
    const float f = __fsub_rn(__uint_as_float(mb), 1.0f);
    float R = -0x1.38c9dep-4f;
    R = __fmaf_rn(R, f, 0x1.055ec6p-3f);
    R = __fmaf_rn(R, f, -0x1.0d8242p-3f);
    R = __fmaf_rn(R, f, 0x1.22d92ep-3f);
    R = __fmaf_rn(R, f, -0x1.54728ap-3f);
    R = __fmaf_rn(R, f, 0x1.99a01cp-3f);
    R = __fmaf_rn(R, f, -0x1.000226p-2f);
    R = __fmaf_rn(R, f, 0x1.555554p-2f);
    const float t = __fmaf_rn(f, R, -0.5f);
    const float lnm = __fmaf_rn(__fmul_rn(f, f), t, f);
    const float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnm));
}

// (sin, cos) of 2 pi v 2^-24, v odd in (0, 2^24)
__device__ __forceinline__ void chan_sincos2pi(uint32_t v, float *sn_out, float *cs_out) {
    const int32_t j = (int32_t)((v + (1u << 21)) >> 22);
    const int32_t ri = (int32_t)v - j * (1 << 22);
    const float r = __fmul_rn(__int2float_rn(ri), 0x1p-24f);
    const float z = __fmul_rn(r, r);
    float S = 0x1.a0b0c6p+8f, C = 0x1.c33bfap+6f;
    S = __fmaf_rn(S, z, -0x1.61b22ap+6f);
    C = __fmaf_rn(C, z, 0x1.b78f76p+5f);
    S = __fmaf_rn(S, z, 0x1.46e1p+6f);
    C = __fmaf_rn(C, z, -0x1.558c8p+6f);
    S = __fmaf_rn(S, z, -0x1.4abc8ap+5f);
    C = __fmaf_rn(C, z, 0x1.03c192p+6f);
    S = __fmaf_rn(S, z, 0x1.921fb6p+2f);
    C = __fmaf_rn(C, z, -0x1.3bd3ccp+4f);
    const float sn = __fmul_rn(r, S);
    const float cs = __fmaf_rn(z, C, 1.0f);
    switch (j & 3) {
        case 0: *sn_out = sn; *cs_out = cs; break;
        case 1: *sn_out = cs; *cs_out = -sn; break;
        case 2: *sn_out = -sn; *cs_out = -cs; break;
        default: *sn_out = -cs; *cs_out = sn; break;
    }
}

// words -> four channel LLRs: Box-Muller pairs (w0, w1) and (w2, w3),
// rho = sqrt(-2 ln u(w0)), g = rho cos(2 pi u(w1)), rho sin(2 pi u(w1)), and
// mu = s2 * fma(sigma, g, x) with s2 = 2 / sigma^2 (binary32 values rounded from double).
// bit e of `bits` is the code bit c of LLR e: BPSK x = 1 - 2c (all-zero codeword: bits = 0)
__device__ __forceinline__ void box_muller_llr(const uint32_t *w, float sigma, float s2, float *mu4,
                                               uint32_t bits = 0u) {
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const uint32_t v0 = 2u * (w[2 * pr] >> 9) + 1u, v1 = 2u * (w[2 * pr + 1] >> 9) + 1u;
        const float u0 = __fmul_rn(__uint2float_rn(v0), 0x1p-24f);
        const float rho = __fsqrt_rn(__fmul_rn(-2.0f, chan_ln(u0)));
        float sn, cs;
        chan_sincos2pi(v1, &sn, &cs);
        const float x0 = ((bits >> (2 * pr)) & 1u) ? -1.0f : 1.0f;
        const float x1 = ((bits >> (2 * pr + 1)) & 1u) ? -1.0f : 1.0f;
        mu4[2 * pr] = __fmul_rn(s2, __fmaf_rn(sigma, __fmul_rn(rho, cs), x0));
        mu4[2 * pr + 1] = __fmul_rn(s2, __fmaf_rn(sigma, __fmul_rn(rho, sn), x1));
    }
}

// four channel LLRs of bits 4q..4q+3 of frame F (code bits in `bits`, LSB = bit 4q)
__device__ __forceinline__ void channel_quad(uint64_t seed, uint64_t F, int q, float sigma, float s2, float *mu4,
                                             uint32_t bits = 0u) {
    uint32_t w[4];
    philox4x32_10((uint32_t)q, (uint32_t)F, (uint32_t)(F >> 32), 0u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    box_muller_llr(w, sigma, s2, mu4, bits);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async; completion by groups)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// blocks of a persistent launch: resident blocks per SM (occupancy API, cached per
// kernel and dynamic shared-memory size) times the SM count; also raises the kernel's
// dynamic shared-memory limit to the largest size requested so far
template <typename K>
int persistent_blocks(K kernel, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void *, size_t> limit;         // kernel -> attribute set
    static std::unordered_map<const void *, std::unordered_map<size_t, int>> cache;  // -> blocks per SM
    static int sms = 0;
    std::lock_guard<std::mutex> lk(mu);
    const void *key = (const void *)kernel;
    auto &per = cache[key];
    auto f = per.find(smem);
    if (f != per.end()) return f->second * sms;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    if (smem > limit[key]) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        limit[key] = smem;
    }
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kWarps * 32, smem);
    if (bps < 1) bps = 1;
    per[smem] = bps;
    return bps * sms;
}

// n / d for a divisor fixed at launch (FastDiv, ldpc_internal.cuh)
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
    const uint32_t t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// arguments of the variable pass in continuous-simulation (refill) mode
struct RefillArgs {
    const uint32_t *sflags = nullptr;  // per package: retire[V], refill[V]
    int *errs = nullptr;               // bit errors of the retiring frames, per slot
    const void *mu = nullptr;          // channel LLRs, frame-major [P][W][N rounded up to 4]
};

__device__ __forceinline__ int sbyte(uint32_t w, int v) { return (int)(int8_t)(uint8_t)(w >> (8 * v)); }

}  // namespace ldpc

namespace ldpc {
// variable pass in refill mode (qc_pipe.cu); sum-product or min-sum, not NOMS
ldpc_status qc_vn_refill(ldpc_code c, const ldpc_decode_opts &o, const RefillArgs &rf, cudaStream_t s);
}  // namespace ldpc

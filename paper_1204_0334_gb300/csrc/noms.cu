// Learned normalized/offset min-sum (NOMS): forward and backward kernels for
// training the per-iteration, per-circulant weights and offsets, over T
// unrolled flooding iterations of Algorithm 1 with the check rule
//   alpha_e = s_e * min(max(w_{l,c(e)} * m_e - o_{l,c(e)}, 0), clip),  m_e = min_{e' != e} |beta_e'|,
// the variable rule of eq. (bpvs) with clipping, and the loss
//   loss = 1/(T N B) sum_l sum_n softplus(-post^(l)_n)
// (BCE of every iteration's posterior against the all-zero codeword).
//
// Layout: packages of 32 V frames, V = 1 for FP32 messages and 2 for binary16 (two
// frames per 32-bit lane word, the FP16 decoder's layout); message buffers [P][E][32]
// lane words (edge order of the block decoder: edge k of block (j, l) is variable
// l*p + k), per-frame FP32 arrays [P][..][32][V].  Betas are kept at checkpoints every
// k iterations in the storage type S (float or half), and so are the alphas; adjoints in
// float.  The backward pass recomputes each segment of k iterations from its checkpoint.
// The forward also keeps every iteration's posteriors: with them and beta^(l) the backward
// variable step needs nothing of alpha^(l), so the check messages are never recomputed.
#include "qc_device.cuh"

#include <algorithm>
#include <vector>

struct ldpc_noms_state {
    int B = 0, T = 0, k = 1, P = 0, msg = LDPC_MSG_F32;
    float clip = 30.0f;
    size_t cap_frames = 0, cap_nck = 0, cap_seg = 0;
    float *mu = nullptr;       // [P][N][32 V]
    void *ping[2] = {nullptr, nullptr};  // non-checkpoint betas (S)
    void *ckpt = nullptr;      // [nck][P][E][32] lane words: beta^(k), beta^(2k), ...
    void *seg = nullptr;       // [k][P][E][32] lane words: recomputed betas of one segment
    float *A = nullptr, *GA = nullptr;  // [P][E][32 V] (A holds lane words)
    // adjoint of beta^(l-1), nonzero only on the two smallest inputs of each row and frame: per
    // row and lane a word of their slots ([P][M][32]: int8 i1, i2 per frame) and their values
    // ([P][M][2][32 V] floats)
    uint32_t *GBs = nullptr;
    float *GBv = nullptr;
    float *posts = nullptr;    // [T][P][N][32 V] (stride N * cap_frames): post^(1..T) of the forward
    size_t cap_T = 0;
    double *acc = nullptr;     // loss: one partial sum per variable-step block, [P][ceil(N / 8)]
    bool have_forward = false;
    const float *params = nullptr;
};

namespace ldpc {

// A lane's 32-bit word of one edge package: one FP32 frame (S = float, packages of
// 32 frames), or two binary16 frames (S = __half, packages of 64 frames, lane l
// holding frames 2l and 2l + 1 -- the FP16 decoder's layout).  Per-frame FP32
// arrays (channel LLRs, posteriors, adjoints) follow the same order:
// [..][32 lanes][V frames].
template <typename S> struct Word;
template <> struct Word<float> {
    static constexpr int V = 1;
    static constexpr uint32_t INF = 0x7f800000u;  // +inf
    static __device__ __forceinline__ void ld(uint32_t w, float *x) { x[0] = __uint_as_float(w); }
    static __device__ __forceinline__ uint32_t pack(const float *x) { return __float_as_uint(x[0]); }
};
template <> struct Word<__half> {
    static constexpr int V = 2;
    static constexpr uint32_t INF = 0x7c007c00u;  // +inf twice
    static __device__ __forceinline__ void ld(uint32_t w, float *x) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        x[0] = f.x;
        x[1] = f.y;
    }
    static __device__ __forceinline__ uint32_t pack(const float *x) {
        const __half2 h = __floats2half2_rn(x[0], x[1]);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
};

// one exponential each: softplus(x) = max(x, 0) + log1p(e^-|x|) (the loss, reported); sigmoid from
// e = e^-|x| and a correctly rounded reciprocal of 1 + e (an adjoint: within an ulp or two)
__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x))); }
__device__ __forceinline__ float sigmoidf(float x) {
    const float e = __expf(-fabsf(x));
    const float r = __frcp_rn(1.0f + e);
    return x >= 0.0f ? r : e * r;
}

// ---------------------------------------------------------------------------
// forward check step: alpha^(l) from beta^(l-1); one warp = one row of one package
// ---------------------------------------------------------------------------
#ifndef NM_FWD_MINB
#define NM_FWD_MINB 5  // resident blocks per SM of the forward check step, rows of up to 24 edges (51 registers)
#endif
// REG: every block of the row is present and L == DCMAX, so the gathers carry no branches
// and all DCMAX loads of a row are in flight together.  Only the two smallest magnitudes,
// the index of the first smallest and the sign bits outlive the gathers: the other edges'
// minimum is mn2 for that index and mn1 for every other edge (on a tie mn2 == mn1).  Lane l
// holds slot l's edge index and the gathers take it by shuffle.  From the channel LLRs
// (FROM_MU, FP32) the frames of a lane word are done one after the other.
template <int DCMAX, typename S, bool FROM_MU, bool REG>
__global__ void __launch_bounds__(kWarps * 32, FROM_MU ? 3 : (DCMAX > 24 ? 4 : NM_FWD_MINB))
nm_cn_fwd(const QcDesc d, const void *__restrict__ bin, uint32_t *__restrict__ A, const float *__restrict__ prm_l,
          float clip, int P) {
    constexpr int V = Word<S>::V;
    __shared__ int s_e[kWarps][32];  // each warp's row: the edge of every slot (-1 absent)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = blockIdx.x * kWarps + warp;
    const int pk = blockIdx.y;
    if (m >= d.M || pk >= P) return;
    const int j = (int)fdiv((uint32_t)m, d.divP), r = m - j * d.p;
    // lane l: the edge of slot l in this row (-1: absent block) and its variable, computed once and
    // broadcast by shuffles
    int my_e = -1, my_n = 0;
    if (REG ? lane < DCMAX : (lane < d.L && d.shift[j * d.L + lane] >= 0)) {
        int k = r + d.shift[j * d.L + lane];
        if (k >= d.p) k -= d.p;
        my_e = d.eoff[j * d.L + lane] + k;
        my_n = lane * d.p + k;
    }
    s_e[warp][lane] = my_e;
    __syncwarp();
    const float2 *prm = reinterpret_cast<const float2 *>(prm_l) + (size_t)j * d.L;
    // the edge of slot l again from the tables (cheap to recompute, unlike a shuffle result that
    // would stay live from the gathers); -1: absent
    auto edge = [&](int l) -> int {
        const int sh = (REG || l < d.L) ? d.shift[j * d.L + l] : -1;
        if (!REG && sh < 0) return -1;
        int k = r + sh;
        if (k >= d.p) k -= d.p;
        return d.eoff[j * d.L + l] + k;
    };
    if constexpr (FROM_MU) {
        const float *mu = reinterpret_cast<const float *>(bin);
#pragma unroll 1
        for (int v = 0; v < V; ++v) {
            float x[DCMAX];
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const int e = __shfl_sync(0xffffffffu, my_e, l);
                const int n = __shfl_sync(0xffffffffu, my_n, l);
                x[l] = (!REG && e < 0) ? INFINITY : mu[(((size_t)pk * d.N + n) * 32 + lane) * V + v];
            }
            uint32_t neg = 0u;
            float mn1 = INFINITY, mn2 = INFINITY;
            int i1 = -1;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const float a = fabsf(x[l]);  // absent edges: +inf, never below mn1
                neg |= (x[l] < 0.0f ? 1u : 0u) << l;
                const bool lo = a < mn1;
                mn2 = lo ? mn1 : fminf(mn2, a);
                i1 = lo ? l : i1;
                mn1 = lo ? a : mn1;
            }
            const uint32_t par = __popc(neg) & 1u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const int e = edge(l);
                if (!REG && e < 0) continue;  // warp-uniform
                const float2 wo = __ldg(prm + l);
                const float mv = l == i1 ? mn2 : mn1;
                const float mag = fminf(fmaxf(fmaf(wo.x, mv, -wo.y), 0.0f), clip);
                const float out = (par ^ ((neg >> l) & 1u)) ? -mag : mag;
                const size_t w = ((size_t)pk * d.E + e) * 32 + lane;
                if constexpr (V == 1) A[w] = __float_as_uint(out);
                else reinterpret_cast<__half *>(A)[w * 2 + v] = __float2half_rn(out);
            }
        }
    } else {
        const uint32_t *bw = reinterpret_cast<const uint32_t *>(bin);
        uint32_t xw[DCMAX];
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            const int e = __shfl_sync(0xffffffffu, my_e, l);
            xw[l] = (!REG && e < 0) ? Word<S>::INF : bw[((size_t)pk * d.E + e) * 32 + lane];
        }
        uint32_t neg[V];
        float mn1[V], mn2[V];
        int i1[V];
        if constexpr (V == 2) {
            // both binary16 frames of a word at once: min and compare are exact on binary16, so the
            // search takes the same decisions as on the FP32 conversions (a < mn1, ties keep the
            // lower slot, -0 is not negative)
            const __half2 inf2 = __half2half2(__ushort_as_half((unsigned short)0x7c00u));
            const __half2 zero2 = __float2half2_rn(0.0f);
            __half2 m1 = inf2, m2 = inf2;
            uint32_t ip = 0xffffffffu, n0 = 0u, n1 = 0u;  // i1 of each frame in 16 bits; sign bits
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const uint32_t x = xw[l], ab = x & 0x7fff7fffu;
                const __half2 a = *reinterpret_cast<const __half2 *>(&ab);
                const uint32_t lo = __hlt2_mask(a, m1);  // 0xffff in each half where a < mn1
                const __half2 t = __hmin2(m2, a);
                const uint32_t m1b = *reinterpret_cast<const uint32_t *>(&m1);
                const uint32_t tb = *reinterpret_cast<const uint32_t *>(&t);
                const uint32_t m2b = (m1b & lo) | (tb & ~lo);
                m2 = *reinterpret_cast<const __half2 *>(&m2b);
                ip = ((uint32_t)l * 0x00010001u & lo) | (ip & ~lo);
                m1 = __hmin2(m1, a);
                const uint32_t ng = x & __hne2_mask(a, zero2) & 0x80008000u;
                n0 |= ((ng >> 15) & 1u) << l;
                n1 |= (ng >> 31) << l;
            }
            const float2 f1 = __half22float2(m1), f2 = __half22float2(m2);
            mn1[0] = f1.x, mn1[1] = f1.y, mn2[0] = f2.x, mn2[1] = f2.y;
            i1[0] = (int)(int16_t)(ip & 0xffffu);
            i1[1] = (int)(int16_t)(ip >> 16);
            neg[0] = n0, neg[1] = n1;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) neg[v] = 0u, mn1[v] = mn2[v] = INFINITY, i1[v] = -1;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                float x[V];
                Word<S>::ld(xw[l], x);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float a = fabsf(x[v]);
                    neg[v] |= (x[v] < 0.0f ? 1u : 0u) << l;
                    const bool lo = a < mn1[v];
                    mn2[v] = lo ? mn1[v] : fminf(mn2[v], a);
                    i1[v] = lo ? l : i1[v];
                    mn1[v] = lo ? a : mn1[v];
                }
            }
        }
        uint32_t par[V];
#pragma unroll
        for (int v = 0; v < V; ++v) par[v] = __popc(neg[v]) & 1u;
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            const int e = s_e[warp][l];  // broadcast read of the row's edge table
            if (!REG && e < 0) continue;  // warp-uniform
            const float2 wo = __ldg(prm + l);
            float out[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float mv = l == i1[v] ? mn2[v] : mn1[v];
                const float mag = fminf(fmaxf(fmaf(wo.x, mv, -wo.y), 0.0f), clip);
                out[v] = (par[v] ^ ((neg[v] >> l) & 1u)) ? -mag : mag;
            }
            A[((size_t)pk * d.E + e) * 32 + lane] = Word<S>::pack(out);
        }
    }
}

// ---------------------------------------------------------------------------
// forward variable step: beta^(l) (clipped, stored as S), posterior, loss term
// ---------------------------------------------------------------------------
template <int JMAX, typename S, bool REG>
__global__ void __launch_bounds__(kWarps * 32)
nm_vn_fwd(const QcDesc d, const uint32_t *__restrict__ A, const float *__restrict__ mu, uint32_t *__restrict__ bout,
          double *__restrict__ acc, float *__restrict__ post, float zinv, float clip, int P, int B) {
    constexpr int V = Word<S>::V;
    __shared__ float red[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = blockIdx.x * kWarps + warp;
    const int pk = blockIdx.y;
    float lsum = 0.0f;
    if (n < d.N && pk < P) {
        const int l = (int)fdiv((uint32_t)n, d.divP), k = n - l * d.p;
        const size_t fb = (((size_t)pk * d.N + n) * 32 + lane) * V;  // this lane's frames, per-frame arrays
        float mv[V];
        if constexpr (V == 1) mv[0] = mu[fb];
        else {
            const float2 m2 = *reinterpret_cast<const float2 *>(mu + fb);
            mv[0] = m2.x;
            mv[1] = m2.y;
        }
        float a[JMAX][V];
        int eid[JMAX];
#pragma unroll
        for (int j = 0; j < JMAX; ++j) {
#pragma unroll
            for (int v = 0; v < V; ++v) a[j][v] = 0.0f;
            eid[j] = -1;
            if (!REG && (j >= d.J || d.shift[j * d.L + l] < 0)) continue;
            eid[j] = d.eoff[j * d.L + l] + k;
            Word<S>::ld(A[((size_t)pk * d.E + eid[j]) * 32 + lane], a[j]);
        }
        float tot[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            tot[v] = mv[v];
#pragma unroll
            for (int j = 0; j < JMAX; ++j) tot[v] += a[j][v];
        }
        if (bout) {
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                if (!REG && eid[j] < 0) continue;
                float out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float s = mv[v];
#pragma unroll
                    for (int j2 = 0; j2 < JMAX; ++j2)
                        if (j2 != j) s += a[j2][v];
                    out[v] = clipf(s, clip);
                }
                bout[((size_t)pk * d.E + eid[j]) * 32 + lane] = Word<S>::pack(out);
            }
        }
        if (post) {
            if constexpr (V == 1) post[fb] = tot[0];
            else *reinterpret_cast<float2 *>(post + fb) = make_float2(tot[0], tot[1]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
            if ((pk * 32 + lane) * V + v < B) lsum += softplusf(-tot[v]) * zinv;
    }
    if (acc) {
        // this block's sum is added to its own partial (the launches of the iterations follow one
        // another on the stream, so no atomic is needed and the total does not depend on timing)
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) red[warp] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += red[w];
            acc[(size_t)blockIdx.y * gridDim.x + blockIdx.x] += s;
        }
    }
}

// ---------------------------------------------------------------------------
// backward variable step: adjoint of alpha^(l) from the loss at iteration l and
// the adjoint of beta^(l) (zero at l = T), through the clip.  What this step needs
// of iteration l is the posterior post^(l), saved by the forward, and where beta^(l)
// stayed inside the clip, read off the stored beta^(l) itself (|beta| < clip exactly
// where the clip was inactive), so alpha^(l) is not recomputed.
// ---------------------------------------------------------------------------
template <int JMAX, typename S, bool REG>
__global__ void __launch_bounds__(kWarps * 32)
nm_vn_bwd(const QcDesc d, const float *__restrict__ post, const uint32_t *__restrict__ bl,
          const uint32_t *__restrict__ gbs, const float *__restrict__ gbv, float *__restrict__ GA, float clip,
          float zinv, int P, int B) {
    constexpr int V = Word<S>::V;
    const int lane = threadIdx.x & 31;
    const int n = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int pk = blockIdx.y;
    if (n >= d.N || pk >= P) return;
    const int l = (int)fdiv((uint32_t)n, d.divP), k = n - l * d.p;
    const size_t fb = (((size_t)pk * d.N + n) * 32 + lane) * V;
    float tot[V];
    if constexpr (V == 1) tot[0] = post[fb];
    else {
        const float2 t2 = *reinterpret_cast<const float2 *>(post + fb);
        tot[0] = t2.x;
        tot[1] = t2.y;
    }
    float gbm[JMAX][V];
    int eid[JMAX];
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
#pragma unroll
        for (int v = 0; v < V; ++v) gbm[j][v] = 0.0f;
        eid[j] = -1;
        if (!REG && (j >= d.J || d.shift[j * d.L + l] < 0)) continue;
        eid[j] = d.eoff[j * d.L + l] + k;
        // the adjoint of beta^(l)_e: nonzero where this edge (slot l of its row) is one of the row's
        // two smallest inputs; it passes the clip only where the clip was inactive
        if (gbs) {
            int r = k - d.shift[j * d.L + l];
            if (r < 0) r += d.p;
            const size_t rw = (size_t)pk * d.M + j * d.p + r;  // the row's record
            // the slots and both values are loaded together (no load waits on another)
            const uint32_t sw = gbs[rw * 32 + lane];
            float g1v[V], g2v[V], b[V];
            if constexpr (V == 1) {
                g1v[0] = gbv[(rw * 2) * 32 + lane];
                g2v[0] = gbv[(rw * 2 + 1) * 32 + lane];
            } else {
                const float2 a1 = *reinterpret_cast<const float2 *>(gbv + (rw * 2) * 64 + lane * 2);
                const float2 a2 = *reinterpret_cast<const float2 *>(gbv + (rw * 2 + 1) * 64 + lane * 2);
                g1v[0] = a1.x, g1v[1] = a1.y, g2v[0] = a2.x, g2v[1] = a2.y;
            }
            Word<S>::ld(bl[((size_t)pk * d.E + eid[j]) * 32 + lane], b);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int s1 = (int)(int8_t)(sw >> (16 * v)), s2 = (int)(int8_t)(sw >> (16 * v + 8));
                const float g = l == s1 ? g1v[v] : (l == s2 ? g2v[v] : 0.0f);
                if (fabsf(b[v]) < clip) gbm[j][v] = g;
            }
        }
    }
    float dpost[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dpost[v] = ((pk * 32 + lane) * V + v < B) ? -sigmoidf(-tot[v]) * zinv : 0.0f;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        if (!REG && eid[j] < 0) continue;
        float g[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            g[v] = dpost[v];
#pragma unroll
            for (int j2 = 0; j2 < JMAX; ++j2)
                if (j2 != j) g[v] += gbm[j2][v];
        }
        const size_t w = ((size_t)pk * d.E + eid[j]) * 32 + lane;
        if constexpr (V == 1) GA[w] = g[0];
        else *reinterpret_cast<float2 *>(GA + w * 2) = make_float2(g[0], g[1]);
    }
}

// ---------------------------------------------------------------------------
// backward check step of iteration 1 (input: the channel LLRs): the parameter
// gradients (beta^(0) = mu needs no adjoint).  m_e = |beta_{e*}| with e* the
// arg-min over the other edges
// (lowest index among ties): e* = idx2 for e = idx1, else idx1; so only the
// two smallest inputs of a row receive gradient.  Persistent warps take items of
// kBwdRows consecutive rows of one block row j, so every row of an item adds to
// the same circulants' gradients: each lane keeps its partial sums per edge slot
// in the warp's slice of dynamic shared memory ([DCMAX][2][32] floats, so that
// three blocks fit per SM) and the warp reduces them once per item (not once per
// row) into block sums in shared memory, flushed once per block.  Lane l holds
// slot l's shift and edge offset; a row's edge indices are computed once per row
// (one per lane) and broadcast by shuffles.  REG: every block of the row is
// present and L == DCMAX (no branches on absent slots).  The frames of a lane
// word (two with binary16 messages) are done one after the other.
// ---------------------------------------------------------------------------
constexpr int kBwdRows = 16;
#ifndef LDPC_NM_BWD_BLOCKS
#define LDPC_NM_BWD_BLOCKS 3
#endif
constexpr int kBwdBlocks = LDPC_NM_BWD_BLOCKS;  // resident blocks per SM of the backward check step

template <int DCMAX, typename S, bool REG>
__global__ void __launch_bounds__(kWarps * 32, kBwdBlocks)
nm_cn_bwd(const QcDesc d, const float *__restrict__ mu, const float *__restrict__ GA, const float *__restrict__ prm_l,
          float *__restrict__ grad_l, float clip, int P) {
    static_assert(DCMAX <= 32, "one lane per edge slot");
    constexpr int V = Word<S>::V;
    __shared__ float sg[kMaxJ * kMaxL * 2];
    extern __shared__ float s_part[];
    for (int i = threadIdx.x; i < d.J * d.L * 2; i += blockDim.x) sg[i] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *part = s_part + (size_t)warp * DCMAX * 2 * 32;  // [l][w or o][lane]
    const int chunks = (d.p + kBwdRows - 1) / kBwdRows;
    const long long total = (long long)P * d.J * chunks;
    for (long long item = (long long)blockIdx.x * kWarps + warp; item < total; item += (long long)gridDim.x * kWarps) {
        const int pk = (int)(item / ((long long)d.J * chunks));
        const int rem = (int)(item - (long long)pk * d.J * chunks);
        const int j = rem / chunks, r0 = (rem - j * chunks) * kBwdRows;
        const int r1 = min(r0 + kBwdRows, d.p);
        const float2 *prm = reinterpret_cast<const float2 *>(prm_l) + (size_t)j * d.L;
        // slot `lane` of this block row: shift (-1 absent) and first edge of its block
        const int my_sh = (lane < DCMAX && (REG || lane < d.L)) ? d.shift[j * d.L + lane] : -1;
        const int my_eo = my_sh >= 0 ? d.eoff[j * d.L + lane] : 0;
        // this lane's partial gradients of (w, o) per edge slot l
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) part[(2 * l) * 32 + lane] = part[(2 * l + 1) * 32 + lane] = 0.0f;
        const size_t base = (size_t)pk * d.E;
        for (int r = r0; r < r1; ++r) {
            // edge of slot `lane` in row r (-1: absent) and its variable
            int my_e = -1, my_n = 0;
            if (REG || my_sh >= 0) {
                int k = r + my_sh;
                if (k >= d.p) k -= d.p;
                my_e = my_eo + k;
                my_n = lane * d.p + k;
            }
#pragma unroll 1
            for (int v = 0; v < V; ++v) {  // the frames of the lane word
            // every load of the row first (beta^(l-1) and the adjoints of alpha^(l) do not depend on
            // each other): one memory round trip per row
            float xin[DCMAX], ga[DCMAX];
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const int e = __shfl_sync(0xffffffffu, my_e, l);
                xin[l] = INFINITY;
                ga[l] = 0.0f;
                if (!REG && e < 0) continue;  // warp-uniform
                const int n = __shfl_sync(0xffffffffu, my_n, l);
                xin[l] = mu[(((size_t)pk * d.N + n) * 32 + lane) * V + v];
                ga[l] = GA[((base + e) * 32 + lane) * V + v];
            }
            // the two smallest magnitudes and their slots (strict <: the lowest index among ties);
            // absent slots hold +inf and never qualify
            uint32_t neg = 0u;
            float mn1 = INFINITY, mn2 = INFINITY;
            int i1 = -1, i2 = -1;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const float a = fabsf(xin[l]);
                neg |= (xin[l] < 0.0f ? 1u : 0u) << l;
                const bool lo1 = a < mn1, lo2 = a < mn2;
                mn2 = lo1 ? mn1 : (lo2 ? a : mn2);
                i2 = lo1 ? i1 : (lo2 ? l : i2);
                mn1 = lo1 ? a : mn1;
                i1 = lo1 ? l : i1;
            }
            const uint32_t par = __popc(neg) & 1u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                if (!REG && ga[l] == 0.0f) continue;  // absent slot, or nothing to propagate
                const float2 wo = __ldg(prm + l);
                const bool first = l == i1;
                const float mv = first ? mn2 : mn1;
                const float sgn = (par ^ ((neg >> l) & 1u)) ? -1.0f : 1.0f;
                const float z = fmaf(wo.x, mv, -wo.y);
                // alpha = s (w m - o) only where that is positive and below the clip
                const bool act = (first ? i2 : i1) >= 0 && z > 0.0f && z < clip;
                if (act) {
                    const float gs = ga[l] * sgn;
                    part[(2 * l) * 32 + lane] = fmaf(gs, mv, part[(2 * l) * 32 + lane]);
                    part[(2 * l + 1) * 32 + lane] -= gs;
                }
            }
            }
        }
        // warp sums of this item's gradients per circulant (j, l)
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            if (!REG && __shfl_sync(0xffffffffu, my_sh, l) < 0) continue;  // warp-uniform
            float gw = part[(2 * l) * 32 + lane], go = part[(2 * l + 1) * 32 + lane];
#pragma unroll
            for (int of = 16; of > 0; of >>= 1) {
                gw += __shfl_xor_sync(0xffffffffu, gw, of);
                go += __shfl_xor_sync(0xffffffffu, go, of);
            }
            if (lane == 0 && (gw != 0.0f || go != 0.0f)) {
                atomicAdd(&sg[(j * d.L + l) * 2], gw);
                atomicAdd(&sg[(j * d.L + l) * 2 + 1], go);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d.J * d.L * 2; i += blockDim.x)
        if (sg[i] != 0.0f) atomicAdd(grad_l + i, sg[i]);
}

// The backward check step for iterations l >= 2 (inputs beta^(l-1) from a message
// store): the same arithmetic as nm_cn_bwd, with the row's inputs staged in shared
// memory.  Each warp keeps the next row's beta words and adjoints of alpha in flight
// in a two-stage ring, copied with cp.async (16 bytes per lane, completion tracked by
// cp.async groups), while it works on the current row out of shared memory; both
// frames of a binary16 lane word are done together, and the partial gradients per
// edge slot stay in registers.  Blocks of four warps, three per SM.
constexpr int kRingWarps = 4;

template <int DCMAX, typename S, bool REG>
__global__ void __launch_bounds__(kRingWarps * 32, 3)
nm_cn_bwd_ring(const QcDesc d, const uint32_t *__restrict__ bw, const float *__restrict__ GA,
               const float *__restrict__ prm_l, uint32_t *__restrict__ gbs, float *__restrict__ gbv,
               float *__restrict__ grad_l, float clip, int P, int want_gb) {
    static_assert(DCMAX <= 32 && DCMAX % 4 == 0, "one lane per edge slot, slots in groups of four");
    constexpr int V = Word<S>::V;
    constexpr int SB = DCMAX * 32;      // words: the beta packages of a row
    constexpr int SG = DCMAX * 32 * V;  // floats: the adjoint packages of a row
    constexpr int STAGE = SB + SG;
    __shared__ float sg[kMaxJ * kMaxL * 2];
    extern __shared__ __align__(16) uint32_t ring_all[];
    for (int i = threadIdx.x; i < d.J * d.L * 2; i += blockDim.x) sg[i] = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *ring = ring_all + (size_t)warp * 2 * STAGE;
    const int chunks = (d.p + kBwdRows - 1) / kBwdRows;
    const long long total = (long long)P * d.J * chunks;
    for (long long item = (long long)blockIdx.x * kRingWarps + warp; item < total;
         item += (long long)gridDim.x * kRingWarps) {
        const int pk = (int)(item / ((long long)d.J * chunks));
        const int rem = (int)(item - (long long)pk * d.J * chunks);
        const int j = rem / chunks, r0 = (rem - j * chunks) * kBwdRows;
        const int r1 = min(r0 + kBwdRows, d.p);
        const float2 *prm = reinterpret_cast<const float2 *>(prm_l) + (size_t)j * d.L;
        // slot `lane` of this block row: shift (-1 absent) and first edge of its block
        const int my_sh = (lane < DCMAX && (REG || lane < d.L)) ? d.shift[j * d.L + lane] : -1;
        const int my_eo = my_sh >= 0 ? d.eoff[j * d.L + lane] : 0;
        const uint32_t pres = __ballot_sync(0xffffffffu, my_sh >= 0);  // present slots (bit l)
        const size_t base = (size_t)pk * d.E;
        // edge of slot `lane` in row r (-1: absent)
        auto row_edge = [&](int r) -> int {
            if (!REG && my_sh < 0) return -1;
            int k = r + my_sh;
            if (k >= d.p) k -= d.p;
            return my_eo + k;
        };
        // starts the copies of row r into stage st
        auto issue = [&](int r, int st) {
            const int me = row_edge(r);
            uint32_t *dst = ring + st * STAGE;
#pragma unroll
            for (int q = 0; q < DCMAX / 4; ++q) {  // beta: 8 chunks of 16 bytes per edge
                const int l = 4 * q + (lane >> 3), sub = lane & 7;
                const int e = __shfl_sync(0xffffffffu, me, l);
                if (REG || e >= 0) cp_async16(dst + l * 32 + sub * 4, bw + (base + e) * 32 + sub * 4);
            }
#pragma unroll
            for (int q = 0; q < DCMAX * V / 4; ++q) {  // adjoints: 8 V chunks per edge
                const int c = 32 * q + lane;
                const int l = c / (8 * V), sub = c - l * (8 * V);
                const int e = __shfl_sync(0xffffffffu, me, l);
                if (REG || e >= 0) cp_async16(dst + SB + l * 32 * V + sub * 4, GA + (base + e) * 32 * V + sub * 4);
            }
            cp_async_commit();
        };
        float pw[DCMAX], po[DCMAX];  // this lane's partial gradients of (w, o) per edge slot
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) pw[l] = po[l] = 0.0f;
        issue(r0, 0);
        for (int r = r0, st = 0; r < r1; ++r, st ^= 1) {
            if (r + 1 < r1) issue(r + 1, st ^ 1);
            else cp_async_commit();  // an empty group: the wait below always leaves one pending
            cp_async_wait<1>();
            __syncwarp();
            const uint32_t *Sb = ring + st * STAGE;
            const float *Sg = reinterpret_cast<const float *>(Sb + SB);
            // the two smallest magnitudes of each frame and their slots (strict <: the lowest index
            // among ties); absent slots never qualify
            uint32_t neg[V];
            float mn1[V], mn2[V];
            int i1[V], i2[V];
#pragma unroll
            for (int v = 0; v < V; ++v) neg[v] = 0u, mn1[v] = mn2[v] = INFINITY, i1[v] = i2[v] = -1;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                if (!REG && !((pres >> l) & 1u)) continue;  // warp-uniform
                float x[V];
                Word<S>::ld(Sb[l * 32 + lane], x);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float a = fabsf(x[v]);
                    neg[v] |= (x[v] < 0.0f ? 1u : 0u) << l;
                    const bool lo1 = a < mn1[v], lo2 = a < mn2[v];
                    mn2[v] = lo1 ? mn1[v] : (lo2 ? a : mn2[v]);
                    i2[v] = lo1 ? i1[v] : (lo2 ? l : i2[v]);
                    mn1[v] = lo1 ? a : mn1[v];
                    i1[v] = lo1 ? l : i1[v];
                }
            }
            uint32_t par[V];
            float g1[V], g2[V];  // adjoints landing on slots i1 and i2
#pragma unroll
            for (int v = 0; v < V; ++v) par[v] = __popc(neg[v]) & 1u, g1[v] = g2[v] = 0.0f;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                if (!REG && !((pres >> l) & 1u)) continue;  // warp-uniform
                const float2 wo = __ldg(prm + l);
                float ga[V];
                if constexpr (V == 1) ga[0] = Sg[l * 32 + lane];
                else {
                    const float2 g = *reinterpret_cast<const float2 *>(Sg + l * 64 + lane * 2);
                    ga[0] = g.x;
                    ga[1] = g.y;
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const bool first = l == i1[v];
                    const float mv = first ? mn2[v] : mn1[v];
                    const float sgn = (par[v] ^ ((neg[v] >> l) & 1u)) ? -1.0f : 1.0f;
                    const float z = fmaf(wo.x, mv, -wo.y);
                    // alpha = s (w m - o) only where that is positive and below the clip
                    if ((first ? i2[v] : i1[v]) >= 0 && z > 0.0f && z < clip) {
                        const float gs = ga[v] * sgn;
                        pw[l] = fmaf(gs, mv, pw[l]);
                        po[l] -= gs;
                        if (first) g2[v] += gs * wo.x;
                        else g1[v] += gs * wo.x;
                    }
                }
            }
            if (want_gb) {
                // sign(beta) of the two smallest inputs (0 for beta = 0)
                float s1[V], s2[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    s1[v] = (i1[v] < 0 || mn1[v] == 0.0f) ? 0.0f : (((neg[v] >> i1[v]) & 1u) ? -1.0f : 1.0f);
                    s2[v] = (i2[v] < 0 || mn2[v] == 0.0f) ? 0.0f : (((neg[v] >> i2[v]) & 1u) ? -1.0f : 1.0f);
                }
                // the adjoint of beta^(l-1) is nonzero on slots i1 and i2 only: one record per row and lane
                const size_t rw = (size_t)pk * d.M + j * d.p + r;
                uint32_t sw = 0u;
#pragma unroll
                for (int v = 0; v < V; ++v)
                    sw |= ((uint32_t)(uint8_t)i1[v] << (16 * v)) | ((uint32_t)(uint8_t)i2[v] << (16 * v + 8));
                gbs[rw * 32 + lane] = sw;
                if constexpr (V == 1) {
                    gbv[(rw * 2) * 32 + lane] = g1[0] * s1[0];
                    gbv[(rw * 2 + 1) * 32 + lane] = g2[0] * s2[0];
                } else {
                    *reinterpret_cast<float2 *>(gbv + (rw * 2) * 64 + lane * 2) = make_float2(g1[0] * s1[0], g1[1] * s1[1]);
                    *reinterpret_cast<float2 *>(gbv + (rw * 2 + 1) * 64 + lane * 2) =
                        make_float2(g2[0] * s2[0], g2[1] * s2[1]);
                }
            }
            __syncwarp();  // the stage is refilled by the next issue
        }
        cp_async_wait<0>();
        // warp sums of this item's gradients per circulant (j, l)
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            if (!REG && !((pres >> l) & 1u)) continue;  // warp-uniform
            float gw = pw[l], go = po[l];
#pragma unroll
            for (int of = 16; of > 0; of >>= 1) {
                gw += __shfl_xor_sync(0xffffffffu, gw, of);
                go += __shfl_xor_sync(0xffffffffu, go, of);
            }
            if (lane == 0 && (gw != 0.0f || go != 0.0f)) {
                atomicAdd(&sg[(j * d.L + l) * 2], gw);
                atomicAdd(&sg[(j * d.L + l) * 2 + 1], go);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d.J * d.L * 2; i += blockDim.x)
        if (sg[i] != 0.0f) atomicAdd(grad_l + i, sg[i]);
}

// the loss: the partial sums added in a fixed order (one block of 1024 threads)
__global__ void __launch_bounds__(1024) nm_loss_out(const double *__restrict__ part, long long np, float *out) {
    __shared__ double sh[1024];
    double t = 0.0;
    for (long long i = threadIdx.x; i < np; i += blockDim.x) t += part[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)sh[0];
}

// partial loss sums of the variable step: one per block of its grid ((N + 7) / 8, P)
static size_t nm_loss_parts(ldpc_code c, const ldpc_noms_state &w) {
    return (size_t)((c->d.N + kWarps - 1) / kWarps) * (w.cap_frames / 32);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static ldpc_status nm_alloc(ldpc_code c, ldpc_noms_state &w, size_t frames, size_t nck, size_t nseg, size_t T) {
    const size_t E = c->d.E, N = c->d.N, M = c->d.M;
    const size_t fr = (frames + 63) / 64 * 64;  // whole packages of 32 or 64 frames
    auto fail = [&]() {
        cudaGetLastError();
        set_error("NOMS workspace allocation failed");
        return LDPC_ENOMEM;
    };
    if (fr > w.cap_frames) {
        cudaDeviceSynchronize();
        cudaFree(w.mu); cudaFree(w.ping[0]); cudaFree(w.ping[1]); cudaFree(w.A); cudaFree(w.GA); cudaFree(w.GBs); cudaFree(w.GBv);
        cudaFree(w.posts); cudaFree(w.ckpt); cudaFree(w.seg); cudaFree(w.acc);
        // nothing is held until every buffer of the new size exists (a failed call leaves no
        // capacity behind that the next call would trust)
        w.mu = w.A = w.GA = w.GBv = w.posts = nullptr;
        w.GBs = nullptr;
        w.ping[0] = w.ping[1] = w.ckpt = w.seg = nullptr;
        w.acc = nullptr;
        w.cap_frames = w.cap_nck = w.cap_seg = w.cap_T = 0;
        const size_t np = (size_t)((N + kWarps - 1) / kWarps) * (fr / 32);
        if (cudaMalloc(&w.mu, N * fr * 4) || cudaMalloc(&w.ping[0], E * fr * 4) || cudaMalloc(&w.ping[1], E * fr * 4) ||
            cudaMalloc(&w.A, E * fr * 4) || cudaMalloc(&w.GA, E * fr * 4) || cudaMalloc(&w.GBs, M * fr * 4) ||
            cudaMalloc(&w.GBv, 2 * M * fr * 4) ||
            cudaMalloc(&w.acc, np * sizeof(double)))
            return fail();
        w.cap_frames = fr;
    }
    if (T > w.cap_T) {
        cudaDeviceSynchronize();
        cudaFree(w.posts);
        w.posts = nullptr;
        w.cap_T = 0;
        if (cudaMalloc(&w.posts, T * N * w.cap_frames * 4)) return fail();
        w.cap_T = T;
    }
    if (nck > w.cap_nck) {
        cudaDeviceSynchronize();
        cudaFree(w.ckpt);
        w.ckpt = nullptr;
        w.cap_nck = 0;
        if (cudaMalloc(&w.ckpt, nck * E * w.cap_frames * 4)) return fail();
        w.cap_nck = nck;
    }
    if (nseg > w.cap_seg) {
        cudaDeviceSynchronize();
        cudaFree(w.seg);
        w.seg = nullptr;
        w.cap_seg = 0;
        if (cudaMalloc(&w.seg, nseg * E * w.cap_frames * 4)) return fail();
        w.cap_seg = nseg;
    }
    return LDPC_OK;
}

// every block of the base matrix is present (the REG kernels)
static bool nm_full(const QcDesc &d) {
    for (int i = 0; i < d.J * d.L; ++i)
        if (d.shift[i] < 0) return false;
    return true;
}

template <typename S>
static ldpc_status nm_step_fwd(ldpc_code c, ldpc_noms_state &w, int l, const void *bin, bool from_mu, void *bout,
                               bool loss, float *post, cudaStream_t s) {
    const QcDesc &d = c->d;
    dim3 cg((d.M + kWarps - 1) / kWarps, w.P), vg((d.N + kWarps - 1) / kWarps, w.P);
    const float *prm = w.params + (size_t)(l - 1) * d.J * d.L * 2;
    const float zinv = (float)(1.0 / ((double)w.T * d.N * w.B));
    const bool full = nm_full(d);
#define NM_CN(DC)                                                                                             \
    do {                                                                                                      \
        if (full && d.L == (DC)) {                                                                            \
            if (from_mu) nm_cn_fwd<DC, S, true, true><<<cg, kWarps * 32, 0, s>>>(d, bin, (uint32_t *)w.A, prm, w.clip, w.P); \
            else nm_cn_fwd<DC, S, false, true><<<cg, kWarps * 32, 0, s>>>(d, bin, (uint32_t *)w.A, prm, w.clip, w.P);        \
        } else if (from_mu) {                                                                                 \
            nm_cn_fwd<DC, S, true, false><<<cg, kWarps * 32, 0, s>>>(d, bin, (uint32_t *)w.A, prm, w.clip, w.P);           \
        } else {                                                                                              \
            nm_cn_fwd<DC, S, false, false><<<cg, kWarps * 32, 0, s>>>(d, bin, (uint32_t *)w.A, prm, w.clip, w.P);          \
        }                                                                                                     \
    } while (0)
    if (d.L <= 8) NM_CN(8);
    else if (d.L <= 16) NM_CN(16);
    else if (d.L <= 24) NM_CN(24);
    else NM_CN(32);
#undef NM_CN
    count_launch();
    if (bout || loss || post) {
        double *acc = loss ? w.acc : nullptr;
        if (full && d.J == 4)
            nm_vn_fwd<4, S, true><<<vg, kWarps * 32, 0, s>>>(d, (const uint32_t *)w.A, w.mu, (uint32_t *)bout, acc, post, zinv, w.clip,
                                                             w.P, w.B);
        else if (d.J <= 4)
            nm_vn_fwd<4, S, false><<<vg, kWarps * 32, 0, s>>>(d, (const uint32_t *)w.A, w.mu, (uint32_t *)bout, acc, post, zinv, w.clip,
                                                              w.P, w.B);
        else
            nm_vn_fwd<8, S, false><<<vg, kWarps * 32, 0, s>>>(d, (const uint32_t *)w.A, w.mu, (uint32_t *)bout, acc, post, zinv, w.clip,
                                                              w.P, w.B);
        count_launch();
    }
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

template <typename S>
static void *ck(ldpc_code c, ldpc_noms_state &w, int idx) {  // checkpoint beta^(idx * k), idx >= 1
    return (char *)w.ckpt + (size_t)(idx - 1) * c->d.E * w.cap_frames * sizeof(S);
}
template <typename S>
static void *sg(ldpc_code c, ldpc_noms_state &w, int idx) {
    return (char *)w.seg + (size_t)idx * c->d.E * w.cap_frames * sizeof(S);
}

static float *nm_post(ldpc_code c, ldpc_noms_state &w, int l) {  // post^(l), l >= 1
    return w.posts + (size_t)(l - 1) * c->d.N * w.cap_frames;
}

template <typename S>
static ldpc_status nm_forward(ldpc_code c, ldpc_noms_state &w, cudaStream_t s) {
    LDPC_CUDA_TRY(cudaMemsetAsync(w.acc, 0, nm_loss_parts(c, w) * sizeof(double), s));
    const void *prev = w.mu;
    bool from_mu = true;
    for (int l = 1; l <= w.T; ++l) {
        void *out;
        if (l == w.T) out = nullptr;  // beta^(T) is never used
        else if (l % w.k == 0) out = ck<S>(c, w, l / w.k);
        else out = w.ping[l & 1];
        ldpc_status st = nm_step_fwd<S>(c, w, l, prev, from_mu, out, true, nm_post(c, w, l), s);
        if (st != LDPC_OK) return st;
        prev = out;
        from_mu = false;
    }
    return LDPC_OK;
}

template <typename S>
static ldpc_status nm_backward(ldpc_code c, ldpc_noms_state &w, float *grad, cudaStream_t s) {
    const QcDesc &d = c->d;
    dim3 vg((d.N + kWarps - 1) / kWarps, w.P);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cb_blocks = std::max(1, sms * kBwdBlocks);  // the resident blocks
    const float zinv = (float)(1.0 / ((double)w.T * d.N * w.B));
    const bool full = nm_full(d);
    int seg_base = -1;  // iterations seg_base+1 .. seg_base+k-1 recomputed into seg
    // beta^(l): the input of the previous (l + 1) step, a checkpoint or a member of the segment
    // that step used -- which is also beta^(l-1)'s segment unless l is a checkpoint, so it is
    // still there
    const void *bnext = nullptr;
    for (int l = w.T; l >= 1; --l) {
        // beta^(l-1): mu, a checkpoint, or a recomputed member of its segment
        const int b = l - 1;
        const void *bin;
        bool from_mu = false;
        if (b == 0) {
            bin = w.mu;
            from_mu = true;
        } else if (b % w.k == 0) {
            bin = ck<S>(c, w, b / w.k);
        } else {
            const int c0 = (b / w.k) * w.k;
            if (seg_base != c0) {
                const void *src = c0 == 0 ? (const void *)w.mu : ck<S>(c, w, c0 / w.k);
                bool fm = c0 == 0;
                for (int q = c0 + 1; q < std::min(c0 + w.k, w.T); ++q) {
                    void *dst = sg<S>(c, w, q - c0 - 1);
                    ldpc_status st = nm_step_fwd<S>(c, w, q, src, fm, dst, false, nullptr, s);
                    if (st != LDPC_OK) return st;
                    src = dst;
                    fm = false;
                }
                seg_base = c0;
            }
            bin = sg<S>(c, w, b - c0 - 1);
        }
        // the adjoints of alpha^(l) (from the saved posteriors and beta^(l)), then of the parameters
        // and beta^(l-1)
        const uint32_t *gbs = l == w.T ? nullptr : w.GBs;  // the adjoint of beta^(T) is zero
        const uint32_t *bl = l == w.T ? nullptr : (const uint32_t *)bnext;
        const float *pl = nm_post(c, w, l);
        if (full && d.J == 4)
            nm_vn_bwd<4, S, true><<<vg, kWarps * 32, 0, s>>>(d, pl, bl, gbs, w.GBv, w.GA, w.clip, zinv, w.P, w.B);
        else if (d.J <= 4)
            nm_vn_bwd<4, S, false><<<vg, kWarps * 32, 0, s>>>(d, pl, bl, gbs, w.GBv, w.GA, w.clip, zinv, w.P, w.B);
        else
            nm_vn_bwd<8, S, false><<<vg, kWarps * 32, 0, s>>>(d, pl, bl, gbs, w.GBv, w.GA, w.clip, zinv, w.P, w.B);
        const float *prm = w.params + (size_t)(l - 1) * d.J * d.L * 2;
        float *gl = grad + (size_t)(l - 1) * d.J * d.L * 2;
        const int want_gb = l > 1;
#define NM_CB1(DC, RG)                                                                                      \
    do {                                                                                                    \
        const size_t psm = (size_t)kWarps * (DC) * 2 * 32 * sizeof(float);                                 \
        auto kfn = nm_cn_bwd<DC, S, RG>;                                                                    \
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);                   \
        kfn<<<cb_blocks, kWarps * 32, psm, s>>>(d, (const float *)bin, w.GA, prm, gl, w.clip, w.P);          \
    } while (0)
#define NM_CR1(DC, RG)                                                                                      \
    do {                                                                                                    \
        const size_t rsm = (size_t)kRingWarps * 2 * ((DC) * 32 * (1 + Word<S>::V)) * 4;                    \
        auto kfn = nm_cn_bwd_ring<DC, S, RG>;                                                               \
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);                   \
        kfn<<<std::max(1, sms) * 3, kRingWarps * 32, rsm, s>>>(d, (const uint32_t *)bin, w.GA, prm, w.GBs,   \
                                                               w.GBv, gl, w.clip, w.P, want_gb);            \
    } while (0)
// iteration 1 reads the channel LLRs (nm_cn_bwd); later ones a message store (nm_cn_bwd_ring)
#define NM_CB(DC)                                  \
    do {                                           \
        const bool rg = full && d.L == (DC);       \
        if (from_mu) {                             \
            if (rg) NM_CB1(DC, true);              \
            else NM_CB1(DC, false);                \
        } else if (rg) {                           \
            NM_CR1(DC, true);                      \
        } else {                                   \
            NM_CR1(DC, false);                     \
        }                                          \
    } while (0)
        if (d.L <= 8) NM_CB(8);
        else if (d.L <= 16) NM_CB(16);
        else if (d.L <= 24) NM_CB(24);
        else NM_CB(32);
#undef NM_CB
#undef NM_CB1
#undef NM_CR1
        count_launch(2);
        LDPC_CUDA_TRY(cudaGetLastError());
        bnext = bin;
    }
    return LDPC_OK;
}

// pack [B][N] -> [P][N][32] with clipping (qc_decode.cu)
ldpc_status pack_frames_w(const float *llr, float *dst, int gamma, int N, float clip, int W, cudaStream_t s);
ldpc_status unpack_frames_w(const float *src, float *dst, int gamma, int N, int W, cudaStream_t s);

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_noms_forward(ldpc_code c, const float *llr, int32_t B, int32_t T, const float *params, int32_t msg,
                              int32_t ckpt_every, float clip, float *loss, float *post, void *stream) {
    if (!c || !llr || B < 1 || T < 1 || !params || !loss || ckpt_every < 1 || !(clip > 0.0f) || clip > 60000.0f ||
        (msg != LDPC_MSG_F32 && msg != LDPC_MSG_F16) || ((uintptr_t)params & 7u)) {
        set_error("need code, llr, B >= 1, T >= 1, params (8-byte aligned), loss, ckpt_every >= 1, 0 < clip <= 60000, "
                  "F32/F16");
        return LDPC_EINVAL;
    }
    if (pointer_kind(llr) != 0 || pointer_kind(params) != 0 || pointer_kind(loss) != 0 ||
        (post && pointer_kind(post) != 0)) {
        set_error("ldpc_noms_forward takes device buffers");
        return LDPC_EINVAL;
    }
    if (c->sparse) {
        set_error("the learned min-sum takes QC codes (parameters per circulant)");
        return LDPC_EUNSUPPORTED;
    }
    if (!c->noms) {
        c->noms = new (std::nothrow) ldpc_noms_state();
        if (!c->noms) {
            set_error("host allocation failed");
            return LDPC_ENOMEM;
        }
    }
    ldpc_noms_state &w = *c->noms;
    w.have_forward = false;  // set again only once this forward has been queued in full
    const int nck = (T - 1) / ckpt_every;
    ldpc_status st =
        nm_alloc(c, w, (size_t)B, (size_t)std::max(nck, 1), (size_t)std::max(ckpt_every - 1, 1), (size_t)T);
    if (st != LDPC_OK) return st;
    w.B = B;
    w.T = T;
    w.k = ckpt_every;
    const int W = msg == LDPC_MSG_F16 ? 64 : 32;  // frames per package: one or two per lane word
    w.P = (B + W - 1) / W;
    w.msg = msg;
    w.clip = clip;
    w.params = params;
    cudaStream_t s = (cudaStream_t)stream;
    st = pack_frames_w(llr, w.mu, B, c->d.N, clip, W, s);
    if (st != LDPC_OK) return st;
    st = msg == LDPC_MSG_F16 ? nm_forward<__half>(c, w, s) : nm_forward<float>(c, w, s);
    if (st != LDPC_OK) return st;
    nm_loss_out<<<1, 1024, 0, s>>>(w.acc, (long long)nm_loss_parts(c, w), loss);
    count_launch();
    if (post) {
        st = unpack_frames_w(nm_post(c, w, T), post, B, c->d.N, W, s);
        if (st != LDPC_OK) return st;
    }
    w.have_forward = true;
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status ldpc_noms_backward(ldpc_code c, const float *params, float *grad, void *stream) {
    if (!c || !params || !grad) {
        set_error("need code, params and grad");
        return LDPC_EINVAL;
    }
    if (!c->noms || !c->noms->have_forward || c->noms->params != params) {
        set_error("ldpc_noms_backward needs the matching ldpc_noms_forward on this code object first");
        return LDPC_EINVAL;
    }
    if (pointer_kind(grad) != 0) {
        set_error("grad must be device memory");
        return LDPC_EINVAL;
    }
    ldpc_noms_state &w = *c->noms;
    cudaStream_t s = (cudaStream_t)stream;
    return w.msg == LDPC_MSG_F16 ? nm_backward<__half>(c, w, grad, s) : nm_backward<float>(c, w, grad, s);
}

}  // extern "C"

namespace ldpc {
void noms_free(ldpc_noms_state *w) {
    if (!w) return;
    cudaFree(w->mu); cudaFree(w->ping[0]); cudaFree(w->ping[1]); cudaFree(w->ckpt); cudaFree(w->seg);
    cudaFree(w->A); cudaFree(w->GA); cudaFree(w->GBs); cudaFree(w->GBv); cudaFree(w->posts); cudaFree(w->acc);
    delete w;
}
}  // namespace ldpc

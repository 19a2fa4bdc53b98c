// Batched BP decoding of QC-LDPC codes on sm_103a (Algorithm 1, Sec. II-B),
// with the device-side channel and error counting of the simulation (Sec. V).
//
// Data layout (HBM).  Frames are grouped in packages of W = 32*V frames; a lane
// owns V consecutive frames and moves 4 bytes per edge (V = 1 float, V = 2
// half, V = 4 int8), so every warp access to one edge is one 128-byte line --
// the paper's Gamma-package idea (Sec. IV-A) at the width of a warp.
//   msg [P][E][W]   edge messages, one store per edge (Sec. IV-A): alpha after
//                   the check pass; after the variable pass beta (F16) or, for
//                   F32 storage, sign(beta) * phi(|beta|), the form the check
//                   pass sums (so each pass evaluates phi once per edge)
//   mu  [P][N][W]   channel LLRs (float; int8 for min-sum)
//   hw  [P][N][V]   hard decisions, one 32-bit word per (variable, frame slot v)
// Edge k of circulant block (j, l) belongs to variable l*p + k, so the check
// pass of row j*p + r reads edge (r + a_jl) mod p of every block of row j and
// the variable pass reads edge k of every block of column l: both are address
// arithmetic on the shift table, with no index tables (LUT_c / LUT_v of Sec.
// IV-A are not needed for QC codes).
#include "ldpc_internal.cuh"
#include "qc_device.cuh"

#include <algorithm>
#include <cstdio>

namespace ldpc {

// ---------------------------------------------------------------------------
// First check-node (horizontal) step, sum-product.  One warp = one check row of
// one package; lane = V frames.  The incoming messages are beta = mu: the
// initialization of Algorithm 1 folded into the first read, so no beta is ever
// written for iteration 0.  Later iterations run the pipelined pass (qc_pipe.cu).
// Sums of phi over the other edges use prefix + suffix sums (the forward-
// backward computation of Sec. IV-A), never "total minus own": that
// subtraction loses the small terms when one input is unreliable.
// ---------------------------------------------------------------------------
template <int DCMAX, int V, bool NOMS>
__global__ void __launch_bounds__(kWarps * 32)
cn_sp_first_kernel(const QcDesc d, uint32_t *__restrict__ msg, const float *__restrict__ mu,
                   const uint32_t *__restrict__ flags, float clip, const float *__restrict__ nparams) {
    constexpr int W = 32 * V;
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int pk = blockIdx.y;
    if (m >= d.M) return;
    const uint32_t *done = flags + (size_t)pk * 5 * V;
    bool lane_on = false, warp_on = false;
    uint32_t act[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        act[v] = ~done[v];
        warp_on |= act[v] != 0;
        lane_on |= (act[v] >> lane) & 1u;
    }
    if (!warp_on) return;

    const int j = m / d.p;
    const int r = m - j * d.p;
    const int *sh = d.shift + j * d.L;
    const int *eo = d.eoff + j * d.L;
    // package-relative bases; offsets below stay in 32 bits (E * 32 < 2^31)
    uint32_t *pmsg = msg + (size_t)pk * d.E * 32 + lane;
    const float *pmu = mu + (size_t)pk * d.N * W + lane * V;
    float ph[DCMAX][V];
    uint32_t neg[V];
#pragma unroll
    for (int v = 0; v < V; ++v) neg[v] = 0u;

    // incoming messages beta = mu
#pragma unroll
    for (int l = 0; l < DCMAX; ++l) {
        const bool on = l < d.L && sh[l] >= 0;
#pragma unroll
        for (int v = 0; v < V; ++v) ph[l][v] = 0.0f;
        if (on) {
            int k = r + sh[l];
            if (k >= d.p) k -= d.p;
            const int n = l * d.p + k;
            float x[V];
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = pmu[n * W + v];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                ph[l][v] = NOMS ? fabsf(x[v]) : phi_f(fabsf(x[v]));
                neg[v] |= (x[v] < 0.0f ? 1u : 0u) << l;
            }
        }
    }
    uint32_t par_all[V];
#pragma unroll
    for (int v = 0; v < V; ++v) par_all[v] = __popc(neg[v]) & 1u;
    if constexpr (NOMS) {
        // normalized/offset min-sum: ph[] holds |beta|; alpha = sign * max(w * m - o, 0)
        float mn1[V], mn2[V];
#pragma unroll
        for (int v = 0; v < V; ++v) mn1[v] = mn2[v] = INFINITY;
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            const bool on = l < d.L && sh[l] >= 0;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!on) ph[l][v] = INFINITY;
                mn2[v] = fminf(mn2[v], fmaxf(mn1[v], ph[l][v]));
                mn1[v] = fminf(mn1[v], ph[l][v]);
            }
        }
        const float *prm = nparams + (size_t)j * d.L * 2;
#pragma unroll
        for (int l = 0; l < DCMAX; ++l) {
            const bool on = l < d.L && sh[l] >= 0;
            if (!on || !lane_on) continue;
            int k = r + sh[l];
            if (k >= d.p) k -= d.p;
            const float w = __ldg(prm + 2 * l), ofs = __ldg(prm + 2 * l + 1);
            float a[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float m = ph[l][v] == mn1[v] ? mn2[v] : mn1[v];
                const float mag = fminf(fmaxf(fmaf(w, m, -ofs), 0.0f), clip);
                a[v] = (par_all[v] ^ ((neg[v] >> l) & 1u)) ? -mag : mag;
            }
            pmsg[(eo[l] + k) * 32] = Lane<V>::pack(a);
        }
        return;
    } else {
        // prefix sums, then the backward sweep adds the suffix sums
        float pre[DCMAX][V];
        {
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.0f;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    pre[l][v] = acc[v];
                    acc[v] += ph[l][v];
                }
        }
        float suf[V];
#pragma unroll
        for (int v = 0; v < V; ++v) suf[v] = 0.0f;
#pragma unroll
        for (int l = DCMAX - 1; l >= 0; --l) {
            const bool on = l < d.L && sh[l] >= 0;
            if (on) {
                int k = r + sh[l];
                if (k >= d.p) k -= d.p;
                float a[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float mag = fminf(phi_f(pre[l][v] + suf[v]), clip);
                    const uint32_t s = par_all[v] ^ ((neg[v] >> l) & 1u);
                    a[v] = s ? -mag : mag;
                }
                if (lane_on) pmsg[(eo[l] + k) * 32] = Lane<V>::pack(a);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) suf[v] += ph[l][v];
        }
    }
}

// ---------------------------------------------------------------------------
// Integer min-sum over int8 messages, 4 frames per lane in one 32-bit word,
// evaluated with the byte-SIMD video instructions.  Check update:
// |alpha_e| = min over the other edges = (|beta_e| == min1) ? min2 : min1 --
// ties give min2 == min1, so no arg-min is needed; the sign is the parity of
// the other signs (sign(0) = +).  Empty extrinsic set: 127.  First iteration
// only (beta = mu); later iterations run the pipelined pass (qc_pipe.cu).
// ---------------------------------------------------------------------------
template <int DCMAX>
__global__ void __launch_bounds__(kWarps * 32)
cn_ms_first_kernel(const QcDesc d, uint32_t *__restrict__ msg, const uint32_t *__restrict__ mu,
                   const uint32_t *__restrict__ flags) {
    constexpr int V = 4;
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int pk = blockIdx.y;
    if (m >= d.M) return;
    const uint32_t *done = flags + (size_t)pk * 5 * V;
    bool lane_on = false, warp_on = false;
    uint32_t act[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        act[v] = ~done[v];
        warp_on |= act[v] != 0;
        lane_on |= (act[v] >> lane) & 1u;
    }
    if (!warp_on) return;
    const int j = m / d.p;
    const int r = m - j * d.p;
    const int *sh = d.shift + j * d.L;
    const int *eo = d.eoff + j * d.L;
    uint32_t ab[DCMAX], sg[DCMAX];
    uint32_t min1 = 0x7f7f7f7fu, min2 = 0x7f7f7f7fu, sgn = 0u;
#pragma unroll
    for (int l = 0; l < DCMAX; ++l) {
        const bool on = l < d.L && sh[l] >= 0;
        ab[l] = 0u;
        sg[l] = 0u;
        if (on) {
            int k = r + sh[l];
            if (k >= d.p) k -= d.p;
            uint32_t x = 0u;
            if (lane_on) x = mu[((size_t)pk * d.N + (size_t)l * d.p + k) * 32 + lane];
            const uint32_t a = __vabsss4(x);
            sg[l] = x & 0x80808080u;
            ab[l] = a;
            sgn ^= sg[l];
            min2 = __vminu4(min2, __vmaxu4(min1, a));
            min1 = __vminu4(min1, a);
        }
    }
    if (!lane_on) return;
#pragma unroll
    for (int l = 0; l < DCMAX; ++l) {
        const bool on = l < d.L && sh[l] >= 0;
        if (!on) continue;
        int k = r + sh[l];
        if (k >= d.p) k -= d.p;
        const uint32_t eq = __vcmpeq4(ab[l], min1);
        const uint32_t mag = (min2 & eq) | (min1 & ~eq);
        const uint32_t s = ((sgn ^ sg[l]) >> 7) & 0x01010101u;  // 1 where the output is negative
        const uint32_t out = __vadd4(mag ^ (s * 0xffu), s);        // two's-complement negate where s
        msg[((size_t)pk * d.E + eo[l] + k) * 32 + lane] = out;
    }
}


// ---------------------------------------------------------------------------
// Syndrome of the current decisions, eq. (hrddcs) checked row by row: bit
// `lane` of flag word `word + v` of a package is set when some check of frame
// (lane, v) is unsatisfied.  One thread per check row; consecutive rows of a
// block row read consecutive hard-decision words (a cyclic shift of one
// column block), and a warp ORs its rows before one atomic per word.
// ---------------------------------------------------------------------------
template <int V>
__global__ void syndrome_kernel(const QcDesc d, const uint32_t *__restrict__ hw, uint32_t *__restrict__ flags,
                                int P, int word) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int pk = blockIdx.y;
    uint32_t syn[V];
#pragma unroll
    for (int v = 0; v < V; ++v) syn[v] = 0u;
    if (m < d.M && pk < P) {
        const int j = m / d.p, r = m - j * d.p;
        for (int l = 0; l < d.L; ++l) {
            const int a = d.shift[j * d.L + l];
            if (a < 0) continue;
            int k = r + a;
            if (k >= d.p) k -= d.p;
            const uint32_t *h = hw + ((size_t)pk * d.N + (size_t)l * d.p + k) * V;
#pragma unroll
            for (int v = 0; v < V; ++v) syn[v] ^= h[v];
        }
    }
    uint32_t *out = flags + (size_t)pk * 5 * V + word;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t any = __reduce_or_sync(0xffffffffu, syn[v]);
        if (any && (threadIdx.x & 31) == 0) atomicOr(out + v, any);
    }
}

// flags init: done = ~valid (padding frames never run), unsat = 0, fin = 0
__global__ void init_flags_kernel(uint32_t *flags, int P, int V, int gamma) {
    const int pk = blockIdx.x * blockDim.x + threadIdx.x;
    if (pk >= P) return;
    uint32_t *b = flags + (size_t)pk * 5 * V;
    const int W = 32 * V;
    for (int v = 0; v < V; ++v) {
        uint32_t valid = 0u;
        for (int ln = 0; ln < 32; ++ln)
            if (pk * W + ln * V + v < gamma) valid |= 1u << ln;
        b[v] = ~valid;
        b[V + v] = 0u;
        b[2 * V + v] = 0u;
        b[3 * V + v] = valid;
        b[4 * V + v] = 0u;
    }
}

// Per-frame finish: frames not stopped early ran max_iter iterations; ok = 1
// iff the last decisions satisfy every check.  Results in package order
// (frame f at iters[f], okv[f]).
__global__ void finish_frames_kernel(const uint32_t *__restrict__ flags, int32_t *__restrict__ iters,
                                     int32_t *__restrict__ okv, int gamma, int V, int max_iter) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= gamma) return;
    const int W = 32 * V;
    const int pk = f / W, ln = (f % W) / V, v = f % V;
    const uint32_t *b = flags + (size_t)pk * 5 * V;
    const bool stopped = (b[v] >> ln) & 1u;  // a valid frame with its done bit set stopped early
    if (!stopped) iters[f] = max_iter;
    okv[f] = ((b[4 * V + v] >> ln) & 1u) ? 0 : 1;
}

// ---------------------------------------------------------------------------
// Frame-major [gamma][N] <-> package layout, through 32x32 shared-memory tiles.
// ---------------------------------------------------------------------------
template <typename Out>
__global__ void pack_llr_kernel(const float *__restrict__ llr, Out *__restrict__ mu, int gamma, int N, int W,
                                int frames_alloc, float clip, float qscale, float pad) {
    __shared__ float tile[32][33];
    const int f0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int f = f0 + i, n = n0 + tx;
        float x = pad;
        if (f < gamma && n < N) x = llr[(size_t)f * N + n];
        tile[i][tx] = x;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += blockDim.y) {
        const int n = n0 + i, f = f0 + tx;
        if (n >= N || f >= frames_alloc) continue;
        const float x = tile[tx][i];
        const size_t idx = ((size_t)(f / W) * N + n) * W + (f % W);
        if (sizeof(Out) == 1) {
            float q = rintf(x * qscale);
            q = fminf(fmaxf(q, -127.0f), 127.0f);
            reinterpret_cast<int8_t *>(mu)[idx] = (int8_t)q;
        } else {
            reinterpret_cast<float *>(mu)[idx] = clipf(x, clip);
        }
    }
}

__global__ void unpack_post_kernel(const float *__restrict__ pk_post, float *__restrict__ post, int gamma, int N,
                                   int W) {
    __shared__ float tile[32][33];
    const int f0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int n = n0 + i, f = f0 + tx;
        float x = 0.0f;
        if (n < N && f < gamma) x = pk_post[((size_t)(f / W) * N + n) * W + (f % W)];
        tile[i][tx] = x;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += blockDim.y) {
        const int f = f0 + i, n = n0 + tx;
        if (f < gamma && n < N) post[(size_t)f * N + n] = tile[tx][i];
    }
}

__global__ void unpack_hard_kernel(const uint32_t *__restrict__ hw, uint8_t *__restrict__ hard, int gamma, int N,
                                   int V) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int W = 32 * V;
    for (int f = blockIdx.y; f < gamma; f += gridDim.y) {
        const int pk = f / W, ln = (f % W) / V, v = f % V;
        hard[(size_t)f * N + n] = (uint8_t)((hw[((size_t)pk * N + n) * V + v] >> ln) & 1u);
    }
}

// ---------------------------------------------------------------------------
// Channel (Sec. V: codeword and noise made on the GPU): all-zero codeword,
// BPSK, AWGN; Philox4x32-10 (Salmon et al., SC'11) + Box-Muller, frame-major
// output [gamma][N] for ldpc_channel.
// ---------------------------------------------------------------------------
__global__ void channel_frames_kernel(float *__restrict__ out, int N, int gamma, uint64_t seed, uint64_t first_frame,
                                      float sigma, float s2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= N) return;
    for (int f = blockIdx.y; f < gamma; f += gridDim.y) {
        float v4[4];
        channel_quad(seed, first_frame + (uint64_t)f, q, sigma, s2, v4);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < N) out[(size_t)f * N + 4 * q + e] = v4[e];
    }
}

// [gamma][N] <-> [P][N][W] for the learned min-sum state (packages of W = 32 or 64 frames;
// frames beyond gamma up to the last package's end are set to +clip)
ldpc_status pack_frames_w(const float *llr, float *dst, int gamma, int N, float clip, int W, cudaStream_t s) {
    const int P = (gamma + W - 1) / W;
    dim3 blk(32, 8), grd((N + 31) / 32, (P * W + 31) / 32);
    count_launch();
    pack_llr_kernel<float><<<grd, blk, 0, s>>>(llr, dst, gamma, N, W, P * W, clip, 1.0f, clip);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status unpack_frames_w(const float *src, float *dst, int gamma, int N, int W, cudaStream_t s) {
    dim3 blk(32, 8), grd((N + 31) / 32, (gamma + 31) / 32);
    count_launch();
    unpack_post_kernel<<<grd, blk, 0, s>>>(src, dst, gamma, N, W);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// the check-node transform on its own, for verification (ldpc_phi_eval)
// variant 0: the decoders' scalar evaluation; 1: CUDA's expm1f/log1pf form; 2: the packed-pair
// evaluation the node passes use (pairs of consecutive elements)
__global__ void phi_eval_kernel(const float *__restrict__ x, float *__restrict__ y, int n, int variant) {
    if (variant == 2) {
        for (int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x); i < n; i += 2 * gridDim.x * blockDim.x) {
            const float x0 = x[i], x1 = i + 1 < n ? x[i + 1] : 1.0f;
            float y0, y1;
            phi2(x0, x1, y0, y1);
            y[i] = y0;
            if (i + 1 < n) y[i + 1] = y1;
        }
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = variant == 0 ? phi_f(x[i]) : phi_ref(x[i]);
}

ldpc_status phi_eval(const float *x, float *y, int n, int variant, cudaStream_t s) {
    const int blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    count_launch();
    phi_eval_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(x, y, n, variant);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

ldpc_status qc_ensure_workspace(ldpc_code c, size_t gamma, int want_host_stage) {
    DecodeWs &w = c->ws;
    const size_t need = round_up(gamma, 128);
    const bool grow = need > w.gamma_cap;
    const bool stage_missing = want_host_stage && !w.stage_llr;
    if (!grow && !stage_missing) return LDPC_OK;
    const size_t cap = grow ? need : w.gamma_cap;
    if (grow) {
        // synchronous reallocation (first use or a larger batch)
        LDPC_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(w.msg);
        cudaFree(w.mu);
        cudaFree(w.post);
        cudaFree(w.hw);
        cudaFree(w.flags);
        cudaFree(w.iters);
        cudaFree(w.counters);
        cudaFree(w.act);
        cudaFree(w.stage_llr);
        cudaFree(w.stage_post);
        cudaFree(w.stage_hard);
        cudaFree(w.stage_i32);
        w = DecodeWs();
        const size_t P32 = cap / 32;
        if (cudaMalloc(&w.msg, (size_t)c->d.E * cap * 4) != cudaSuccess ||
            cudaMalloc(&w.mu, (size_t)c->d.N * cap * 4) != cudaSuccess ||
            cudaMalloc(&w.post, (size_t)c->d.N * cap * 4) != cudaSuccess ||
            cudaMalloc(&w.hw, (size_t)c->d.N * P32 * 4) != cudaSuccess ||
            cudaMalloc(&w.flags, P32 * 5 * 4) != cudaSuccess ||
            cudaMalloc(&w.iters, cap * 2 * 4) != cudaSuccess ||
            cudaMalloc(&w.counters, 8 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&w.act, (P32 + 1) * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation for %zu frames failed", cap);
            return LDPC_ENOMEM;
        }
        w.gamma_cap = cap;
        w.msg_bytes = (size_t)c->d.E * cap * 4;
    }
    if (want_host_stage && !w.stage_llr) {
        if (cudaMalloc(&w.stage_llr, (size_t)c->d.N * cap * 4) != cudaSuccess ||
            cudaMalloc(&w.stage_post, (size_t)c->d.N * cap * 4) != cudaSuccess ||
            cudaMalloc(&w.stage_hard, (size_t)c->d.N * cap) != cudaSuccess ||
            cudaMalloc(&w.stage_i32, cap * 2 * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("device staging allocation for %zu frames failed", cap);
            return LDPC_ENOMEM;
        }
    }
    return LDPC_OK;
}

static int words_per_lane(const ldpc_decode_opts &o) { return lanes_per_word(o.msg); }

ldpc_status qc_pack_llr(ldpc_code c, const float *llr, int gamma, const ldpc_decode_opts &o, cudaStream_t s) {
    const int V = words_per_lane(o), W = 32 * V;
    const int P = (gamma + W - 1) / W;
    dim3 blk(32, 8), grd((c->d.N + 31) / 32, (P * W + 31) / 32);
    count_launch();
    if (o.algo == LDPC_ALGO_MS) {
        pack_llr_kernel<int8_t><<<grd, blk, 0, s>>>(llr, (int8_t *)c->ws.mu, gamma, c->d.N, W, P * W, 0.0f,
                                                    ldexpf(1.0f, o.frac_bits), 1e30f);
    } else {
        pack_llr_kernel<float><<<grd, blk, 0, s>>>(llr, (float *)c->ws.mu, gamma, c->d.N, W, P * W, o.clip, 1.0f,
                                                   o.clip);
    }
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

template <int DCMAX, int V, bool NOMS>
static void launch_cn_first(ldpc_code c, int P, const ldpc_decode_opts &o, cudaStream_t s) {
    dim3 grd((c->d.M + kWarps - 1) / kWarps, P);
    // F32 sum-product storage carries sign(beta) * phi(|beta|) between the passes; F16 and
    // NOMS carry beta (FP16's range cannot hold phi of reliable messages)
    cn_sp_first_kernel<DCMAX, V, NOMS><<<grd, kWarps * 32, 0, s>>>(
        c->d, (uint32_t *)c->ws.msg, (const float *)c->ws.mu, c->ws.flags, o.clip, o.noms_params);
}
template <int DCMAX>
static void launch_cn_ms_first(ldpc_code c, int P, cudaStream_t s) {
    dim3 grd((c->d.M + kWarps - 1) / kWarps, P);
    cn_ms_first_kernel<DCMAX><<<grd, kWarps * 32, 0, s>>>(c->d, (uint32_t *)c->ws.msg,
                                                         (const uint32_t *)c->ws.mu, c->ws.flags);
}

template <int DCMAX>
static void cn_first_dispatch(ldpc_code c, int P, const ldpc_decode_opts &o, cudaStream_t s) {
    if (o.algo == LDPC_ALGO_MS) launch_cn_ms_first<DCMAX>(c, P, s);
    else if (o.algo == LDPC_ALGO_NOMS) {
        if (o.msg == LDPC_MSG_F16) launch_cn_first<DCMAX, 2, true>(c, P, o, s);
        else launch_cn_first<DCMAX, 1, true>(c, P, o, s);
    } else if (o.msg == LDPC_MSG_F16) launch_cn_first<DCMAX, 2, false>(c, P, o, s);
    else launch_cn_first<DCMAX, 1, false>(c, P, o, s);
}

ldpc_status qc_syndrome(ldpc_code c, int P, int V, int word, cudaStream_t s) {
    dim3 grd((c->d.M + 255) / 256, P);
    if (V == 1) syndrome_kernel<1><<<grd, 256, 0, s>>>(c->d, c->ws.hw, c->ws.flags, P, word);
    else if (V == 2) syndrome_kernel<2><<<grd, 256, 0, s>>>(c->d, c->ws.hw, c->ws.flags, P, word);
    else syndrome_kernel<4><<<grd, 256, 0, s>>>(c->d, c->ws.hw, c->ws.flags, P, word);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status qc_decode_device(ldpc_code c, int gamma, const ldpc_decode_opts &o, bool want_post, cudaStream_t s) {
    if (c->sparse) return sparse_decode_device(c, gamma, o, want_post, s);
    const int V = words_per_lane(o), W = 32 * V;
    const int P = (gamma + W - 1) / W;
    init_flags_kernel<<<(P + 127) / 128, 128, 0, s>>>(c->ws.flags, P, V, gamma);
    LDPC_CUDA_TRY(cudaMemsetAsync(c->ws.hw, 0, (size_t)P * c->d.N * V * 4, s));
    ldpc_status st = qc_compact(c, P, V, s);  // every package starts active
    if (st != LDPC_OK) return st;
    count_launch(4);  // init, compact, final syndrome, finish
    const int dcm = c->d.dc_max;
    for (int it = 1; it <= o.max_iter; ++it) {
        const bool syn = o.early_stop && it >= 2;
        const int par = it & 1;
        const int slot_cn = prof_begin(0, s);
        if (it == 1) {
            // beta = mu: the first check pass reads the channel LLRs
            if (dcm <= 8) cn_first_dispatch<8>(c, P, o, s);
            else if (dcm <= 16) cn_first_dispatch<16>(c, P, o, s);
            else if (dcm <= 24) cn_first_dispatch<24>(c, P, o, s);
            else cn_first_dispatch<32>(c, P, o, s);
        } else {
            // early stop: the syndrome of the decisions after it-1 complete iterations (never before the first), then the check pass
            if (syn) {
                st = qc_syndrome(c, P, V, (1 + par) * V, s);
                if (st != LDPC_OK) return st;
                count_launch();
            }
            st = qc_cn_pipe(c, o, it, s);
            if (st != LDPC_OK) return st;
        }
        prof_end(slot_cn, s);
        const int slot_vn = prof_begin(1, s);
        st = qc_vn_pipe(c, o, syn, want_post, it, par, s);
        if (st != LDPC_OK) return st;
        prof_end(slot_vn, s);
        count_launch(2);
        if (o.early_stop && it < o.max_iter) {
            st = qc_compact(c, P, V, s);
            if (st != LDPC_OK) return st;
            count_launch();
        }
    }
    st = qc_syndrome(c, P, V, 4 * V, s);  // fin words: the last decisions
    if (st != LDPC_OK) return st;
    finish_frames_kernel<<<(gamma + 255) / 256, 256, 0, s>>>(c->ws.flags, c->ws.iters,
                                                             c->ws.iters + c->ws.gamma_cap, gamma, V, o.max_iter);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// flag words of a fresh decode of gamma frames (padding frames start stopped)
ldpc_status qc_init_flags(ldpc_code c, int gamma, int V, cudaStream_t s) {
    const int P = (gamma + 32 * V - 1) / (32 * V);
    init_flags_kernel<<<(P + 127) / 128, 128, 0, s>>>(c->ws.flags, P, V, gamma);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// syndrome of the last decisions, iteration counts and ok flags of every frame
// iteration counts and ok flags of every frame from the flag words (the fin words must hold
// the syndrome of the last decisions)
ldpc_status qc_finish_frames(ldpc_code c, int gamma, const ldpc_decode_opts &o, cudaStream_t s) {
    finish_frames_kernel<<<(gamma + 255) / 256, 256, 0, s>>>(c->ws.flags, c->ws.iters, c->ws.iters + c->ws.gamma_cap,
                                                             gamma, words_per_lane(o), o.max_iter);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status qc_finish(ldpc_code c, int gamma, const ldpc_decode_opts &o, cudaStream_t s) {
    const int V = words_per_lane(o);
    const int P = (gamma + 32 * V - 1) / (32 * V);
    ldpc_status st = qc_syndrome(c, P, V, 4 * V, s);
    if (st != LDPC_OK) return st;
    finish_frames_kernel<<<(gamma + 255) / 256, 256, 0, s>>>(c->ws.flags, c->ws.iters, c->ws.iters + c->ws.gamma_cap,
                                                             gamma, V, o.max_iter);
    count_launch(2);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status qc_unpack_outputs(ldpc_code c, int gamma, const ldpc_decode_opts &o, float *post, uint8_t *hard,
                              int32_t *iters, int32_t *ok, cudaStream_t s) {
    const int V = words_per_lane(o), W = 32 * V;
    if (iters) LDPC_CUDA_TRY(cudaMemcpyAsync(iters, c->ws.iters, (size_t)gamma * 4, cudaMemcpyDeviceToDevice, s));
    if (ok)
        LDPC_CUDA_TRY(cudaMemcpyAsync(ok, c->ws.iters + c->ws.gamma_cap, (size_t)gamma * 4, cudaMemcpyDeviceToDevice,
                                      s));
    if (post) {
        dim3 blk(32, 8), grd((c->d.N + 31) / 32, (gamma + 31) / 32);
        count_launch();
        unpack_post_kernel<<<grd, blk, 0, s>>>(c->ws.post, post, gamma, c->d.N, W);
    }
    if (hard) {
        dim3 grd((c->d.N + 255) / 256, gamma < 65535 ? gamma : 65535);
        count_launch();
        unpack_hard_kernel<<<grd, 256, 0, s>>>(c->ws.hw, hard, gamma, c->d.N, V);
    }
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status qc_channel_frames(ldpc_code c, double sigma, uint64_t seed, uint64_t first_frame, int gamma, float *out,
                              cudaStream_t s) {
    const int Q = (c->d.N + 3) / 4;
    dim3 grd((Q + 127) / 128, gamma < 65535 ? gamma : 65535);
    count_launch();
    channel_frames_kernel<<<grd, 128, 0, s>>>(out, c->d.N, gamma, seed, first_frame, (float)sigma,
                                              (float)(2.0 / (sigma * sigma)));
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}


}  // namespace ldpc

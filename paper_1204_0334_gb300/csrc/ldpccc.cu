// Pipelined BP decoder of the LDPC convolutional code derived from a QC base
// (Sec. II-D unwrapping, Algorithm 2, Sec. IV-B), Gamma streams at once.
//
// Code.  Lambda = gcd(J, L); a frame holds c = (L/Lambda) p variables, a check
// layer (J/Lambda) p checks.  Layer R (type a = R mod Lambda) holds base block
// rows j = a*Jb .. a*Jb + Jb - 1; base block column l (frame type l / Lb)
// connects it to frame F = R - ((a - l/Lb) mod Lambda), i.e. to frames
// R - ms .. R with ms = Lambda - 1 (the sub-block H_{a, b} of H_QC).  Frames
// with negative index do not exist (start-up, Sec. IV-B-2 step 3).
//
// Schedule (Algorithm 2).  At slot t frame t enters; processor i (1..I)
// updates check layer t - (i-1)(ms+1), then every processor updates frame
// t - (i-1)(ms+1) - ms; the frame leaving processor I is decided.  All I
// layers go in one check-pass launch and all I frames in one variable-pass
// launch (Sec. IV-B-3: "processed in parallel").
//
// Time-invariant variant (ldpccc_create_tanner): the polynomial parity-check matrix
// [D^{a_jl}] -- check j at time instant t meets bit l at instant t - a_jl.  Frames of
// p instants (c = L p, layers of J p checks, one frame type) give a memory-1 code: check
// (j, tau) of layer R meets bit (l, tau - a) of frame R when tau >= a, else bit
// (l, tau - a + p) of frame R - 1.  Algorithm 2 runs unchanged with ms = 1.
//
// Memory (the "moving processors" of Sec. IV-B-2: relabelling, no copies).
// Frame F lives in ring slot F mod (I*Lambda) from its arrival until its
// decision; its channel LLRs in mu[slot][P][c][32] and its J*c edge messages in
// msg[slot][P][J*c][32], edge (j, ll, k) of block (j, l = b*Lb + ll) at
// (j*Lb + ll)*p + k.  Between the passes an edge holds alpha (after the check
// pass) or sign(beta)*phi(|beta|) (after the variable pass).  Processor 1's
// layer sees no frame that has been through a variable pass yet (frame R - d
// gets its first one at slot R - d + ms >= R), so it reads the channel LLRs
// straight from the ring: the edges of an arriving frame need no initial fill.
#include "qc_device.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

struct ldpccc_s {
    ldpc::QcDesc d;          // base code
    int lam, Jb, Lb, c, cb, ms, I, gamma, P, ring;  // lam: frames between processors (ms + 1)
    int types = 1;           // frame / layer types (period): Lambda, or 1 for the time-invariant code
    int tanner = 0;          // 1: delays D^{a_jl} instead of the sub-block unwrapping
    int device = 0;
    long long t = 0;         // next slot (= index of the next frame to enter)
    float *mu = nullptr;     // [ring][P][c][32]
    uint32_t *msg = nullptr; // [ring][P][J*c][32]
    float *stage = nullptr;  // host-staging of an input window [gamma][T][c]
    size_t stage_cap = 0;
    uint8_t *hstage = nullptr;
    float *pstage = nullptr;
};

namespace ldpc {

struct CcDesc {
    int lam, Jb, Lb, c, cb, ms, I, P, ring, Ef;
    int tanner;  // per-edge frame lag from the row and the delay (time-invariant code)
};

__device__ __forceinline__ int mod_pos(long long x, int m) {
    long long r = x % m;
    return (int)(r < 0 ? r + m : r);
}

// frames t0 .. t0+T-1 of [gamma][T][c] into the ring, clipped
__global__ void cc_enter_kernel(const float *__restrict__ llr, float *__restrict__ mu, CcDesc g, int gamma, int T,
                                int tt, long long t, float clip) {
    __shared__ float tile[32][33];
    const int v0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += blockDim.y) {
        const int s = s0 + i, v = v0 + tx;
        tile[i][tx] = (s < gamma && v < g.c) ? llr[((size_t)s * T + tt) * g.c + v] : clip;
    }
    __syncthreads();
    const int slot = mod_pos(t, g.ring);
    for (int i = ty; i < 32; i += blockDim.y) {
        const int v = v0 + i, s = s0 + tx;
        if (v >= g.c || s >= g.P * 32) continue;
        mu[(((size_t)slot * g.P + s / 32) * g.c + v) * 32 + (s % 32)] = clipf(tile[tx][i], clip);
    }
}

constexpr int kCcStages = 3;  // ring slots per warp
// consecutive check rows per check-pass work item: up to 32 edges (one lane each)
__host__ __device__ constexpr int cc_rows(int dcmax) { return dcmax <= 8 ? 4 : (dcmax <= 16 ? 2 : 1); }
constexpr int kCcNV = 4;      // consecutive variables per variable-pass work item

__device__ __forceinline__ int wrap_lam(int x, int lam) { return x < 0 ? x + lam : x; }

// per-slot constants: t clamped to 2^30 (only compared with frame lags below I*Lambda + Lambda),
// t mod ring, layer type a = t mod Lambda, and the variable pass's frame type (t - ms) mod Lambda
struct SlotC {
    int t, tm, a, bv;
};

// launch geometry: item counts and their divisors
struct CcGeo {
    FastDiv RB, Jb, P, G, p;  // row blocks per block row, Jb, packages, variable groups, p
};

// Check pass of slot t over processors 0 .. n_i - 1 (layers R = t - i*Lambda >= 0).  Work
// items are (processor, package, block row, cc_rows(DCMAX) consecutive rows); persistent warps walk
// them with the items' cc_rows(DCMAX) * DCMAX 128-byte edge packages copied into the warp's shared
// ring by cp.async two items ahead.  The layer's type a = t mod Lambda is the same for every
// processor, so base column l meets frame F = R - ((a - l / Lb) mod Lambda) in ring slot
// (t mod ring - i*Lambda - that lag) mod ring.  Processor 1 reads its edges' beta = mu from
// the channel ring (no frame has had a variable pass yet); the others read
// sign(beta) * phi(|beta|) as the variable pass stored it.
template <int DCMAX>
__global__ void __launch_bounds__(kWarps * 32)
cc_cn_pipe_kernel(const QcDesc d, CcDesc g, CcGeo q, uint32_t *__restrict__ msg, const float *__restrict__ mu,
                  SlotC sc, float clip, int n_i) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_sh[kMaxJ * kMaxL], s_eb[kMaxJ * kMaxL], s_ll[kMaxL], s_dl[kMaxL];
    for (int x = threadIdx.x; x < d.J * d.L; x += blockDim.x) {
        const int j = x / d.L, l = x - j * d.L;
        const int b = l / g.Lb, ll = l - b * g.Lb;
        s_sh[x] = d.shift[x];
        s_eb[x] = (j * g.Lb + ll) * d.p;  // first edge of block (j, l) within a frame
        if (j == 0) {
            s_ll[l] = ll;
            s_dl[l] = wrap_lam(sc.a - b, g.lam);  // frame lag of base column l
        }
    }
    __syncthreads();
    constexpr int ROWS = cc_rows(DCMAX);
    constexpr int NE = ROWS * DCMAX;  // edges of an item
    constexpr int WORDS = NE * 32;
    static_assert(NE <= 32, "one lane per edge of an item");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kCcStages * WORDS;
    const int per_i = (int)(q.P.d * q.Jb.d * q.RB.d);
    const int total = n_i * per_i;  // the host keeps I * P * cb below 2^31
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;

    struct Item {
        int i, pk, j, r0;
    };
    auto geo = [&](int it) {
        Item o;
        uint32_t x = (uint32_t)it;
        const uint32_t x1 = fdiv(x, q.RB);
        o.r0 = (int)(x - x1 * q.RB.d) * ROWS;
        const uint32_t x2 = fdiv(x1, q.Jb);
        const int jj = (int)(x1 - x2 * q.Jb.d);
        const uint32_t x3 = fdiv(x2, q.P);
        o.pk = (int)(x2 - x3 * q.P.d);
        o.i = (int)x3;
        o.j = sc.a * g.Jb + jj;
        return o;
    };
    // package line read for edge e = rr * DCMAX + l of an item (channel ring for processor 1)
    // and the message line written, or -1 where the edge is absent
    auto edge = [&](const Item &o, int e, int &src, int &dstl) {
        src = dstl = -1;
        const int rr = e / DCMAX, l = e - rr * DCMAX;
        const int r = o.r0 + rr;
        if (l >= d.L || r >= d.p) return;
        const int sh = s_sh[o.j * d.L + l];
        if (sh < 0) return;
        int back = o.i * g.lam + s_dl[l];  // t - F
        int k;
        if (g.tanner) {  // bit instant tau - a, in the previous frame when negative
            k = r - sh;
            if (k < 0) k += d.p, ++back;
        } else {
            k = r + sh;
            if (k >= d.p) k -= d.p;
        }
        if (back > sc.t) return;  // frame not yet arrived
        int fs = sc.tm - back;
        if (fs < 0) fs += g.ring;
        dstl = (fs * g.P + o.pk) * g.Ef + s_eb[o.j * d.L + l] + k;
        src = o.i == 0 ? (fs * g.P + o.pk) * g.c + s_ll[l] * d.p + k : dstl;
    };

    auto issue = [&](int it, int slot) -> int {
        int mine = -1;
        if (it < total) {
            const Item o = geo(it);
            uint32_t *dst = ring + slot * WORDS;
            const uint32_t *base = o.i == 0 ? reinterpret_cast<const uint32_t *>(mu) : msg;
            const int grp = lane >> 3, sub = lane & 7;
            // lane e < NE looks up edge e once (the line it reads and the one it writes); the
            // copies take the read lines by shuffle
            int my_src = -1;
            if (lane < NE) edge(o, lane, my_src, mine);
#pragma unroll
            for (int e0 = 0; e0 < NE; e0 += 4) {
                const int e = e0 + grp;
                const int src = __shfl_sync(0xffffffffu, my_src, e & 31);
                if ((NE % 4 == 0 || e < NE) && src >= 0)
                    cp_async16(dst + e * 32 + sub * 4, base + (size_t)src * 32 + sub * 4);
            }
        }
        cp_async_commit();
        return mine;
    };

    int offr[kCcStages];
#pragma unroll
    for (int s = 0; s < kCcStages - 1; ++s) offr[s] = issue(item + s * GW, s);
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kCcStages - 1] = issue(item + (kCcStages - 1) * GW, (slot + kCcStages - 1) % kCcStages);
        cp_async_wait<kCcStages - 1>();
        __syncwarp();
        const uint32_t *S = ring + slot * WORDS;
        const int myoff = offr[0];
#pragma unroll
        for (int s = 0; s < kCcStages - 1; ++s) offr[s] = offr[s + 1];
        const bool p1 = item < per_i;  // processor 1 (warp-uniform)
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr) {
            float xs[DCMAX];
            uint32_t sgn = 0u, pres = 0u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                xs[l] = 0.0f;
                if (__shfl_sync(0xffffffffu, myoff, rr * DCMAX + l) >= 0) {
                    xs[l] = __uint_as_float(S[(rr * DCMAX + l) * 32 + lane]);
                    sgn ^= __float_as_uint(xs[l]);
                    pres |= 1u << l;
                }
            }
            if (pres == 0u) continue;  // row past p (warp-uniform)
            if (p1) {  // channel LLRs: transform here (absent edges stay 0)
#pragma unroll
                for (int l = 0; l < DCMAX; ++l)
                    if ((pres >> l) & 1u) xs[l] = with_sign_of(phi_f(fabsf(xs[l])), xs[l]);
            }
            float pre[DCMAX];
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                pre[l] = acc;
                acc += fabsf(xs[l]);
            }
            // phi of two edges' sums per packed evaluation, in the suffix sums' descending order
            static_assert(DCMAX % 2 == 0, "edge pairs");
            float suf = 0.0f;
#pragma unroll
            for (int l = DCMAX - 1; l >= 1; l -= 2) {
                const float a0 = pre[l] + suf;
                suf += fabsf(xs[l]);
                const float a1 = pre[l - 1] + suf;
                suf += fabsf(xs[l - 1]);
                float m0, m1;
                phi2(a0, a1, m0, m1);
                const int o0 = __shfl_sync(0xffffffffu, myoff, rr * DCMAX + l);
                const int o1 = __shfl_sync(0xffffffffu, myoff, rr * DCMAX + l - 1);
                if (o0 >= 0)
                    msg[(size_t)o0 * 32 + lane] =
                        __float_as_uint(fminf(m0, clip)) | ((sgn ^ __float_as_uint(xs[l])) & 0x80000000u);
                if (o1 >= 0)
                    msg[(size_t)o1 * 32 + lane] =
                        __float_as_uint(fminf(m1, clip)) | ((sgn ^ __float_as_uint(xs[l - 1])) & 0x80000000u);
            }
        }
        __syncwarp();
        slot = (slot + 1) % kCcStages;
    }
    cp_async_wait<0>();
}

// Variable pass of slot t over processors 0 .. n_i - 1 (frames F = t - i*Lambda - ms >= 0);
// items are (processor, package, kCcNV consecutive variables).  Every processor's frame has
// type b = (t - ms) mod Lambda and sits in ring slot (t mod ring - i*Lambda - ms) mod ring.
// The frame leaving processor I (i = I - 1) gets its posterior and hard decision at output
// position q_out.
template <int JMAX>
__global__ void __launch_bounds__(kWarps * 32)
cc_vn_pipe_kernel(const QcDesc d, CcDesc g, CcGeo q, uint32_t *__restrict__ msg, const float *__restrict__ mu,
                  SlotC sc, float clip, int n_i, int gamma, int T_out, int q_out, uint8_t *__restrict__ hard,
                  float *__restrict__ post) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_sh[kMaxJ * kMaxL];
    for (int x = threadIdx.x; x < d.J * d.L; x += blockDim.x) s_sh[x] = d.shift[x];
    __syncthreads();
    constexpr int MU = 0, AL = kCcNV * 32, WORDS = AL + kCcNV * JMAX * 32;
    static_assert(kCcNV == 4 && kCcNV * JMAX <= 32, "item layout");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kCcStages * WORDS;
    const int per_i = (int)(q.P.d * q.G.d);
    const int total = n_i * per_i;
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;

    struct Geo {
        int i, pk, v0, fs, ll0, k0;
    };
    auto geo = [&](int it) {
        Geo o;
        uint32_t x = (uint32_t)it;
        const uint32_t x1 = fdiv(x, q.G);
        o.v0 = (int)(x - x1 * q.G.d) * kCcNV;
        const uint32_t x2 = fdiv(x1, q.P);
        o.pk = (int)(x1 - x2 * q.P.d);
        o.i = (int)x2;
        int fs = sc.tm - o.i * g.lam - g.ms;
        if (fs < 0) fs += g.ring;
        if (fs < 0) fs += g.ring;
        o.fs = fs;
        o.ll0 = (int)fdiv((uint32_t)o.v0, q.p);
        o.k0 = o.v0 - o.ll0 * d.p;
        return o;
    };
    // message line of edge (variable v0 + iv of the item's frame, block row j), or -1
    auto eline = [&](const Geo &o, int iv, int j) -> int {
        if (o.v0 + iv >= g.c || j >= d.J) return -1;
        int ll = o.ll0, k = o.k0 + iv;
        if (k >= d.p) k -= d.p, ++ll;
        if (s_sh[j * d.L + sc.bv * g.Lb + ll] < 0) return -1;
        return (o.fs * g.P + o.pk) * g.Ef + (j * g.Lb + ll) * d.p + k;
    };

    auto issue = [&](int it, int slot) -> int {
        int mine = -1;
        if (it < total) {
            const Geo o = geo(it);
            uint32_t *dst = ring + slot * WORDS;
            const int grp = lane >> 3, sub = lane & 7;
            if (o.v0 + grp < g.c)  // one channel line per lane group
                cp_async16(dst + MU + grp * 32 + sub * 4,
                           reinterpret_cast<const uint32_t *>(mu) +
                               ((size_t)(o.fs * g.P + o.pk) * g.c + o.v0 + grp) * 32 + sub * 4);
            // lane tt looks up edge (variable tt / JMAX, row tt % JMAX) once; the copies take it by shuffle
            if (lane < kCcNV * JMAX) mine = eline(o, lane / JMAX, lane % JMAX);
#pragma unroll
            for (int qq = 0; qq < JMAX; ++qq) {
                const int tt = 4 * qq + grp;
                const int e = __shfl_sync(0xffffffffu, mine, tt & 31);
                if (e >= 0) cp_async16(dst + AL + tt * 32 + sub * 4, msg + (size_t)e * 32 + sub * 4);
            }
        }
        cp_async_commit();
        return mine;
    };

    int offr[kCcStages];
#pragma unroll
    for (int s = 0; s < kCcStages - 1; ++s) offr[s] = issue(item + s * GW, s);
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kCcStages - 1] = issue(item + (kCcStages - 1) * GW, (slot + kCcStages - 1) % kCcStages);
        cp_async_wait<kCcStages - 1>();
        __syncwarp();
        const uint32_t *S = ring + slot * WORDS;
        const int myoff = offr[0];
#pragma unroll
        for (int s = 0; s < kCcStages - 1; ++s) offr[s] = offr[s + 1];
        const uint32_t x1 = fdiv((uint32_t)item, q.G);
        const int v0 = (int)((uint32_t)item - x1 * q.G.d) * kCcNV;
        const uint32_t x2 = fdiv(x1, q.P);
        const int pk = (int)(x1 - x2 * q.P.d);
        const bool out_here = (int)x2 == g.I - 1 && q_out >= 0;
        const int sidx = pk * 32 + lane;
#pragma unroll
        for (int iv = 0; iv < kCcNV; ++iv) {
            const int v = v0 + iv;
            if (v >= g.c) break;  // warp-uniform
            const float m = __uint_as_float(S[MU + iv * 32 + lane]);
            float a[JMAX];
            int e[JMAX];
            float tot = m;
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                e[j] = __shfl_sync(0xffffffffu, myoff, iv * JMAX + j);
                a[j] = e[j] >= 0 ? __uint_as_float(S[AL + (iv * JMAX + j) * 32 + lane]) : 0.0f;
                tot += a[j];
            }
            // store sign(beta) * phi(|beta|), beta = clip(sm); phi on packed pairs of edges
            float sm[JMAX], ph[JMAX];
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                sm[j] = m;
#pragma unroll
                for (int j2 = 0; j2 < JMAX; ++j2)
                    if (j2 != j) sm[j] += a[j2];
            }
#pragma unroll
            for (int j = 0; j + 1 < JMAX; j += 2)
                phi_fin2(fminf(fabsf(sm[j]), clip), fminf(fabsf(sm[j + 1]), clip), ph[j], ph[j + 1]);
            if (JMAX % 2) ph[JMAX - 1] = phi_fin(fminf(fabsf(sm[JMAX - 1]), clip));
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
                if (e[j] < 0) continue;  // warp-uniform
                msg[(size_t)e[j] * 32 + lane] = __float_as_uint(with_sign_of(ph[j], sm[j]));
            }
            if (out_here && sidx < gamma) {
                const float pst = clipf(tot, clip);
                const size_t oi = ((size_t)sidx * T_out + q_out) * g.c + v;
                if (hard) hard[oi] = pst < 0.0f ? 1 : 0;
                if (post) post[oi] = pst;
            }
        }
        __syncwarp();
        slot = (slot + 1) % kCcStages;
    }
    cp_async_wait<0>();
}

// channel LLRs of frames first .. first+T-1 of every stream: all-zero frames over
// BPSK/AWGN; bit n of frame f of stream s draws from Philox counter (n/4, f mod 2^32,
// s, 1) under key (seed mod 2^32, seed / 2^32)
__global__ void cc_channel_kernel(float *__restrict__ out, int gamma, int T, int c, long long first, uint64_t seed,
                                  float sigma, float s2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= c) return;
    for (int st = blockIdx.y; st < gamma * T; st += gridDim.y) {
        const int s = st / T, tt = st - s * T;
        const uint64_t f = (uint64_t)(first + tt);
        uint32_t w[4];
        philox4x32_10((uint32_t)q, (uint32_t)f, (uint32_t)s, 1u, (uint32_t)seed, (uint32_t)(seed >> 32), w);
        float v4[4];
        box_muller_llr(w, sigma, s2, v4);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < c) out[((size_t)s * T + tt) * c + 4 * q + e] = v4[e];
    }
}

static CcDesc cc_desc(const ldpccc_s *cc) {
    return CcDesc{cc->lam, cc->Jb, cc->Lb, cc->c, cc->cb, cc->ms, cc->I, cc->P, cc->ring, cc->d.J * cc->c,
                  cc->tanner};
}

static SlotC slot_consts(const ldpccc_s *cc, long long t) {
    SlotC c;
    c.t = (int)std::min<long long>(t, 1ll << 30);
    c.tm = (int)(t % cc->ring);
    c.a = (int)(t % cc->types);
    c.bv = (int)(((t - cc->ms) % cc->types + cc->types) % cc->types);
    return c;
}

static CcGeo cc_geo(const ldpccc_s *cc, int rows) {
    CcGeo q;
    q.RB = fast_div((uint32_t)((cc->d.p + rows - 1) / rows));
    q.Jb = fast_div((uint32_t)cc->Jb);
    q.P = fast_div((uint32_t)cc->P);
    q.G = fast_div((uint32_t)((cc->c + kCcNV - 1) / kCcNV));
    q.p = fast_div((uint32_t)cc->d.p);
    return q;
}

template <int DCMAX>
static void cc_cn_launch(const ldpccc_s *cc, const CcDesc &g, long long t, float clip, int n_i, cudaStream_t s) {
    auto k = cc_cn_pipe_kernel<DCMAX>;
    const size_t smem = (size_t)kWarps * kCcStages * cc_rows(DCMAX) * DCMAX * 32 * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(cc->d, g, cc_geo(cc, cc_rows(DCMAX)), cc->msg, cc->mu, slot_consts(cc, t), clip,
                                        n_i);
}

template <int JMAX>
static void cc_vn_launch(const ldpccc_s *cc, const CcDesc &g, long long t, float clip, int n_i, int T_out, int q,
                         uint8_t *hard, float *post, cudaStream_t s) {
    auto k = cc_vn_pipe_kernel<JMAX>;
    const size_t smem = (size_t)kWarps * kCcStages * (kCcNV + kCcNV * JMAX) * 32 * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(cc->d, g, cc_geo(cc, 1), cc->msg, cc->mu, slot_consts(cc, t), clip, n_i,
                                        cc->gamma, T_out, q, hard, post);
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

static ldpc_status cc_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                             bool tanner, ldpccc *out) {
    if (!out) {
        set_error("out is NULL");
        return LDPC_EINVAL;
    }
    *out = nullptr;
    if (I < 1 || gamma < 1) {
        set_error("need I >= 1 processors and gamma >= 1 streams");
        return LDPC_EINVAL;
    }
    ldpc_code base = nullptr;
    ldpc_status st = ldpc_code_create(shifts, J, L, p, &base);
    if (st != LDPC_OK) return st;
    ldpccc cc = new (std::nothrow) ldpccc_s();
    if (!cc) {
        ldpc_code_destroy(base);
        set_error("host allocation failed");
        return LDPC_ENOMEM;
    }
    cc->d = base->d;
    ldpc_code_destroy(base);
    if (tanner) {
        int amax = 0;
        for (int x = 0; x < J * L; ++x) amax = std::max(amax, (int)shifts[x]);
        cc->tanner = 1;
        cc->types = 1;
        cc->Jb = J;
        cc->Lb = L;
        cc->ms = amax > 0 ? 1 : 0;
        cc->lam = cc->ms + 1;
    } else {
        cc->types = std::gcd(J, L);
        cc->Jb = J / cc->types;
        cc->Lb = L / cc->types;
        cc->ms = cc->types - 1;
        cc->lam = cc->types;
    }
    cc->c = cc->Lb * p;
    cc->cb = cc->Jb * p;
    cc->I = I;
    cc->gamma = gamma;
    cc->P = (gamma + 31) / 32;
    cc->ring = I * cc->lam;
    // the passes index 128-byte package lines and work items with 32-bit integers
    if ((long long)cc->ring * cc->P * J * cc->c >= (1ll << 31) || (long long)I * cc->P * J * cc->c >= (1ll << 31)) {
        const long long lines = (long long)cc->ring * cc->P * J * cc->c;
        delete cc;
        set_error("I * (ms + 1) * ceil(gamma / 32) * J * c = %lld package lines exceeds 2^31", lines);
        return LDPC_EINVAL;
    }
    cudaGetDevice(&cc->device);
    const size_t mu_b = (size_t)cc->ring * cc->P * cc->c * 32 * 4;
    const size_t msg_b = (size_t)cc->ring * cc->P * J * cc->c * 32 * 4;
    if (cudaMalloc(&cc->mu, mu_b) != cudaSuccess || cudaMalloc(&cc->msg, msg_b) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(cc->mu);
        cudaFree(cc->msg);
        delete cc;
        set_error("device allocation of the %zu-byte ring failed", mu_b + msg_b);
        return LDPC_ENOMEM;
    }
    *out = cc;
    return LDPC_OK;
}

ldpc_status ldpccc_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                          ldpccc *out) {
    return cc_create(shifts, J, L, p, I, gamma, false, out);
}

ldpc_status ldpccc_create_tanner(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                                 ldpccc *out) {
    return cc_create(shifts, J, L, p, I, gamma, true, out);
}

ldpc_status ldpccc_destroy(ldpccc cc) {
    if (!cc) return LDPC_OK;
    cudaFree(cc->mu);
    cudaFree(cc->msg);
    cudaFree(cc->stage);
    cudaFree(cc->hstage);
    cudaFree(cc->pstage);
    delete cc;
    return LDPC_OK;
}

ldpc_status ldpccc_dims(ldpccc cc, int32_t *c, int32_t *b, int32_t *ms, int32_t *lambda) {
    if (!cc) {
        set_error("ldpccc is NULL");
        return LDPC_EINVAL;
    }
    if (c) *c = cc->c;
    if (b) *b = cc->c - cc->cb;
    if (ms) *ms = cc->ms;
    if (lambda) *lambda = cc->types;
    return LDPC_OK;
}

ldpc_status ldpccc_reset(ldpccc cc) {
    if (!cc) {
        set_error("ldpccc is NULL");
        return LDPC_EINVAL;
    }
    cc->t = 0;
    return LDPC_OK;
}

ldpc_status ldpccc_decode_window(ldpccc cc, const float *llr, int32_t T, float clip, uint8_t *hard, float *post,
                                 int64_t *first_out, int32_t *n_out, void *stream) {
    if (!cc || !llr || T < 1 || !n_out || !(clip > 0.0f)) {
        set_error("need ldpccc, llr, T >= 1, n_out and clip > 0");
        return LDPC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)cc->gamma * T * cc->c;
    const bool host_in = pointer_kind(llr) == 1;
    const bool host_hard = hard && pointer_kind(hard) == 1;
    const bool host_post = post && pointer_kind(post) == 1;
    if ((host_in || host_hard || host_post) && cc->stage_cap < nb) {
        LDPC_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(cc->stage);
        cudaFree(cc->hstage);
        cudaFree(cc->pstage);
        cc->stage = nullptr;
        cc->hstage = nullptr;
        cc->pstage = nullptr;
        cc->stage_cap = 0;
        if (cudaMalloc(&cc->stage, nb * 4) != cudaSuccess || cudaMalloc(&cc->hstage, nb) != cudaSuccess ||
            cudaMalloc(&cc->pstage, nb * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("staging allocation failed");
            return LDPC_ENOMEM;
        }
        cc->stage_cap = nb;
    }
    const float *src = llr;
    if (host_in) {
        LDPC_CUDA_TRY(cudaMemcpyAsync(cc->stage, llr, nb * 4, cudaMemcpyHostToDevice, s));
        src = cc->stage;
    }
    uint8_t *dh = host_hard ? cc->hstage : hard;
    float *dp = host_post ? cc->pstage : post;
    const CcDesc g = cc_desc(cc);
    // frames decided in this window: t - I*Lambda + 1 for t = t0 .. t0 + T - 1
    const long long t0 = cc->t;
    const long long first_dec = t0 - (long long)cc->ring + 1;
    int n = 0;
    const int dcm = cc->d.L;
    dim3 eblk(32, 8), egrd((cc->c + 31) / 32, cc->P);
    for (int tt = 0; tt < T; ++tt) {
        const long long t = t0 + tt;
        cc_enter_kernel<<<egrd, eblk, 0, s>>>(src, cc->mu, g, cc->gamma, T, tt, t, clip);
        // processors whose layer (check pass) / frame (variable pass) exists yet
        const int n_cn = (int)std::min<long long>(cc->I, t / cc->lam + 1);
        const int n_vn = t < cc->ms ? 0 : (int)std::min<long long>(cc->I, (t - cc->ms) / cc->lam + 1);
        if (dcm <= 4) cc_cn_launch<4>(cc, g, t, clip, n_cn, s);
        else if (dcm <= 6) cc_cn_launch<6>(cc, g, t, clip, n_cn, s);
        else if (dcm <= 8) cc_cn_launch<8>(cc, g, t, clip, n_cn, s);
        else if (dcm <= 16) cc_cn_launch<16>(cc, g, t, clip, n_cn, s);
        else if (dcm <= 24) cc_cn_launch<24>(cc, g, t, clip, n_cn, s);
        else cc_cn_launch<32>(cc, g, t, clip, n_cn, s);
        const long long Fd = t - (long long)cc->ring + 1;  // frame decided at this slot
        const int q = Fd >= 0 ? (int)(Fd - (first_dec > 0 ? first_dec : 0)) : -1;
        if (q >= 0) ++n;
        if (n_vn > 0) {
            if (cc->d.J == 3) cc_vn_launch<3>(cc, g, t, clip, n_vn, T, q, dh, dp, s);
            else if (cc->d.J <= 4) cc_vn_launch<4>(cc, g, t, clip, n_vn, T, q, dh, dp, s);
            else cc_vn_launch<8>(cc, g, t, clip, n_vn, T, q, dh, dp, s);
        }
        count_launch(n_vn > 0 ? 3 : 2);
    }
    LDPC_CUDA_TRY(cudaGetLastError());
    cc->t = t0 + T;
    // the decided frames land at output positions 0 .. n-1 of each stream's [T][c] block
    if (host_hard || host_post) {
        for (int sidx = 0; sidx < cc->gamma && n > 0; ++sidx) {
            const size_t off = (size_t)sidx * T * cc->c;
            if (host_hard) LDPC_CUDA_TRY(cudaMemcpyAsync(hard + off, dh + off, (size_t)n * cc->c, cudaMemcpyDeviceToHost, s));
            if (host_post)
                LDPC_CUDA_TRY(cudaMemcpyAsync(post + off, dp + off, (size_t)n * cc->c * 4, cudaMemcpyDeviceToHost, s));
        }
    }
    *n_out = n;
    if (first_out) *first_out = n > 0 ? (first_dec > 0 ? first_dec : 0) : -1;
    return LDPC_OK;
}

ldpc_status ldpccc_channel(ldpccc cc, double ebn0_db, uint64_t seed, int64_t first_frame, int32_t T,
                           float *llr_out, void *stream) {
    if (!cc || !llr_out || T < 1 || first_frame < 0 || !std::isfinite(ebn0_db)) {
        set_error("need ldpccc, llr_out, T >= 1, first_frame >= 0 and a finite Eb/N0");
        return LDPC_EINVAL;
    }
    if (pointer_kind(llr_out) != 0) {
        set_error("ldpccc_channel writes device memory");
        return LDPC_EINVAL;
    }
    const double R = (double)(cc->c - cc->cb) / cc->c;
    if (!(R > 0.0)) {
        set_error("rate b/c is not positive");
        return LDPC_EINVAL;
    }
    const double sigma = std::sqrt(1.0 / (2.0 * R * std::pow(10.0, ebn0_db / 10.0)));
    const int Q = (cc->c + 3) / 4;
    const long long rows = (long long)cc->gamma * T;
    dim3 grd((Q + 127) / 128, rows < 65535 ? (unsigned)rows : 65535u);
    count_launch();
    cc_channel_kernel<<<grd, 128, 0, (cudaStream_t)stream>>>(llr_out, cc->gamma, T, cc->c, first_frame, seed,
                                                            (float)sigma, (float)(2.0 / (sigma * sigma)));
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"

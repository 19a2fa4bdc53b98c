// Software-pipelined check-node and variable-node passes (Algorithm 1,
// horizontal and vertical steps) for the QC block-code decoder.
//
// The node passes stream the message store through HBM.  Each warp needs the
// 128-byte packages of 24 edges (check pass) or of 4 variables x J edges plus
// their channel LLRs (variable pass) before it can compute, and then spends a
// long stretch on arithmetic: with one work item per warp the SM runs out of
// bytes in flight.  Here warps are persistent: each walks a strided list of
// work items and keeps the packages of its next items in flight in
// its own shared-memory ring, copied with cp.async (16 bytes per lane,
// completion tracked by cp.async groups -- hardware waits, no spinning), while
// it computes the current item out of shared memory.  Results go straight to
// global memory (in place, Sec. IV-A).  Only packages with a frame still
// running are visited: a compaction pass after each variable pass lists them.
#include "qc_device.cuh"


namespace ldpc {

#ifndef LDPC_CN_STAGES
#define LDPC_CN_STAGES 3
#endif
#ifndef LDPC_VN_STAGES
#define LDPC_VN_STAGES 3
#endif
constexpr int kCnStages = LDPC_CN_STAGES;  // ring slots per warp, check pass
constexpr int kVnStages = LDPC_VN_STAGES;  // ring slots per warp, variable pass
constexpr int kModeSP = 0, kModeMS = 1, kModeNOMS = 2;
constexpr int kNV = 4;  // consecutive variables per variable-pass work item
constexpr int kNomsSmemTable = 48 << 10;  // largest learned-parameter table kept in shared memory

template <int DCMAX>
struct CnStage {
    static constexpr int SEG = DCMAX * 32;  // edge packages, [l][32 words]
    static constexpr int FL = SEG;          // done words [V], fresh-frame words [V] (V <= 4)
    static constexpr int WORDS = SEG + 8;
};

// ---------------------------------------------------------------------------
// check pass (iterations >= 2): sum-product, learned normalized/offset
// min-sum, or integer min-sum.  REG: every block of the row is present and
// L == DCMAX (regular QC code).  The message offsets of an item's DCMAX edges
// stay in registers (lane l holds edge l's, broadcast with a shuffle), so the
// ring holds only message packages and three blocks of eight warps fit on an SM.
// ---------------------------------------------------------------------------
// SPARSE: a general code (index tables; edges of a row are consecutive)
// (register budgets: three blocks per SM for one-frame lane words, two otherwise)
template <int DCMAX, int V, bool XF, int MODE, bool REG, bool SPARSE = false>
__global__ void __launch_bounds__(kWarps * 32, (V == 1 ? 3 : 2))
cn_pipe_kernel(const QcDesc d, uint32_t *__restrict__ msg, const uint32_t *__restrict__ flags,
               const uint32_t *__restrict__ fresh, const int *__restrict__ act, float clip,
               const float *__restrict__ nparams, const int *__restrict__ ages, int T, SparseTab tab) {
    static_assert(!(SPARSE && (REG || MODE == kModeNOMS)), "general codes: irregular rows, no learned min-sum");
    const int LB = SPARSE ? DCMAX : d.L;  // bound of the edge index within a row
    using St = CnStage<DCMAX>;
    // learned min-sum with frames at different iterations (continuous simulation): each lane's
    // frames pick their own parameter row from their iteration counts, staged after the packages
    constexpr int W = 32 * V;
    constexpr int RW = St::WORDS + (MODE == kModeNOMS ? W : 0);
    // the parameter table [T][J*L] (w, o) in shared memory after the rings, rows padded to
    // S = 1 mod 16 pairs so that lanes reading different rows fall in different banks
    const int PS = ((d.J * d.L + 14) / 16) * 16 + 1;
    const bool prm_smem = MODE == kModeNOMS && ages && T * PS * 8 <= kNomsSmemTable;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_sh[kMaxJ * kMaxL], s_eo[kMaxJ * kMaxL];
    for (int i = threadIdx.x; i < d.J * d.L; i += blockDim.x) {
        s_sh[i] = d.shift[i];
        s_eo[i] = d.eoff[i];
    }
    float2 *s_prm = reinterpret_cast<float2 *>(smem + kWarps * kCnStages * RW);
    if (prm_smem) {
        for (int x = threadIdx.x; x < T * d.J * d.L; x += blockDim.x) {
            const int row = x / (d.J * d.L), c = x - row * (d.J * d.L);
            s_prm[row * PS + c] = reinterpret_cast<const float2 *>(nparams)[x];
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kCnStages * RW;
    // work items (package, check row); the host keeps packages * rows below 2^31
    const int total = act[0] * d.M;
    const int *list = act + 1;
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;

    // starts the copies of item `it` into ring slot `slot`; returns this lane's
    // edge offset (lane l < DCMAX: edge l of the row, in 32-word packages; -1 if absent)
    auto issue = [&](int it, int slot) -> int {
        int mine = -1;
        if (it < total) {
            const int a = (int)fdiv((uint32_t)it, d.divM);
            const int m = it - a * d.M;
            const int pk = __ldg(list + a);
            const uint32_t *gmsg = msg + (size_t)pk * d.E * 32;
            uint32_t *dst = ring + slot * RW;
            const int g = lane >> 3, sub = lane & 7;
            if constexpr (SPARSE) {
                const int e0 = __ldg(tab.rp + m), deg = __ldg(tab.rp + m + 1) - e0;
#pragma unroll
                for (int q = 0; q < DCMAX / 4; ++q) {
                    const int l = 4 * q + g;
                    if (l < deg) cp_async16(dst + l * 32 + sub * 4, gmsg + (size_t)(e0 + l) * 32 + sub * 4);
                }
                if (lane < deg) mine = e0 + lane;
                if (lane < V) cp_async4(dst + St::FL + lane, flags + (size_t)pk * 5 * V + lane);
                cp_async_commit();
                return mine;
            }
            const int j = (int)fdiv((uint32_t)m, d.divP), r = m - j * d.p;
            if (MODE == kModeNOMS && ages) {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    cp_async4(dst + St::WORDS + lane * V + v, ages + (size_t)pk * W + lane * V + v);
            }
            // lane l computes edge l's offset once; the copies take it by shuffle
            if (lane < DCMAX && (REG || lane < d.L)) {
                const int sh = s_sh[j * d.L + lane];
                if (REG || sh >= 0) {
                    int k = r + sh;
                    if (k >= d.p) k -= d.p;
                    mine = s_eo[j * d.L + lane] + k;
                }
            }
#pragma unroll
            for (int q = 0; q < DCMAX / 4; ++q) {
                const int l = 4 * q + g;
                const int o = __shfl_sync(0xffffffffu, mine, l);
                if (REG || o >= 0) cp_async16(dst + l * 32 + sub * 4, gmsg + (size_t)o * 32 + sub * 4);
            }
            if (lane < V) cp_async4(dst + St::FL + lane, flags + (size_t)pk * 5 * V + lane);
            else if (fresh && lane < 2 * V) cp_async4(dst + St::FL + lane, fresh + (size_t)pk * 2 * V + lane);
        }
        cp_async_commit();
        return mine;
    };

    int offr[kCnStages];
#pragma unroll
    for (int s = 0; s < kCnStages - 1; ++s) offr[s] = issue(item + s * GW, s);
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kCnStages - 1] = issue(item + (kCnStages - 1) * GW, (slot + kCnStages - 1) % kCnStages);
        cp_async_wait<kCnStages - 1>();
        __syncwarp();
        const uint32_t *S = ring + slot * RW;
        const int myoff = offr[0];
#pragma unroll
        for (int s = 0; s < kCnStages - 1; ++s) offr[s] = offr[s + 1];
        const int pk = __ldg(list + fdiv((uint32_t)item, d.divM));
        uint32_t *gmsg = msg + (size_t)pk * d.E * 32 + lane;
        bool lane_on = false;
        // frames that entered their slot this step (continuous simulation): alpha = 0, so the
        // variable pass that follows starts them at beta = mu (initialization of Alg. 1)
        bool fr[V];
        uint32_t frmask = 0u, keep[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            lane_on |= ((~S[St::FL + v]) >> lane) & 1u;
            fr[v] = fresh && ((S[St::FL + V + v] >> lane) & 1u);
            keep[v] = fr[v] ? 0u : 0xffffffffu;
            if (fr[v]) frmask |= 0xffu << (8 * v);
        }
        if constexpr (MODE == kModeSP) {
            // xs: signed terms sign(beta) * phi(|beta|) (XF: as stored by the variable pass);
            // the output sign is the XOR of the other edges' sign bits
            float xs[DCMAX][V];
            uint32_t sgn[V];
#pragma unroll
            for (int v = 0; v < V; ++v) sgn[v] = 0u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
#pragma unroll
                for (int v = 0; v < V; ++v) xs[l][v] = 0.0f;
                if (REG || (l < LB && __shfl_sync(0xffffffffu, myoff, l) >= 0)) {
                    float x[V];
                    Lane<V>::unpack(S[l * 32 + lane], x);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        xs[l][v] = XF ? x[v] * XfScale<V>::load : copysignf(phi_f(fabsf(x[v])), x[v]);
                        sgn[v] ^= __float_as_uint(x[v]);
                    }
                }
            }
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
                        acc[v] += fabsf(xs[l][v]);
                    }
            }
            float suf[V];
#pragma unroll
            for (int v = 0; v < V; ++v) suf[v] = 0.0f;
            // two edges (V = 1) or the two frames of a lane word (V = 2) per packed phi evaluation,
            // in the same descending order as the suffix sums
#pragma unroll
            for (int l = DCMAX - 1; l >= 0; l -= (V == 1 ? 2 : 1)) {
                float arg[2][V], mag[2][V];
#pragma unroll
                for (int h = 0; h < (V == 1 ? 2 : 1); ++h)
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        arg[h][v] = pre[l - h][v] + suf[v];
                        suf[v] += fabsf(xs[l - h][v]);
                    }
                if constexpr (V == 1) phi2(arg[0][0], arg[1][0], mag[0][0], mag[1][0]);
                else phi2(arg[0][0], arg[0][1], mag[0][0], mag[0][1]);
#pragma unroll
                for (int h = 0; h < (V == 1 ? 2 : 1); ++h) {
                    const int le = l - h;
                    const int o = __shfl_sync(0xffffffffu, myoff, le);
                    if (REG || o >= 0) {
                        float out[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const float m = fminf(mag[h][v], clip);
                            // |alpha| with the XOR of the other edges' signs; 0 for a frame that has
                            // just entered its slot
                            out[v] = __uint_as_float(
                                (__float_as_uint(m) | ((sgn[v] ^ __float_as_uint(xs[le][v])) & 0x80000000u)) &
                                keep[v]);
                        }
                        if (lane_on) gmsg[(size_t)o * 32] = Lane<V>::pack(out);
                    }
                }
            }
        } else if constexpr (MODE == kModeNOMS) {
            // normalized/offset min-sum: alpha = sign * max(w * m - o, 0), (w, o) of this
            // iteration and circulant (j, l); m = min over the other edges = (|beta| == min1 ? min2 : min1)
            const int j = (int)fdiv((uint32_t)(item - (int)fdiv((uint32_t)item, d.divM) * d.M), d.divP);
            // parameter rows: this launch's iteration, or per frame (row = iterations run - 1)
            const float2 *prm[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                int row = 0;
                if (ages) row = min(max((int)S[St::WORDS + lane * V + v] - 1, 0), T - 1);
                prm[v] = prm_smem ? s_prm + row * PS + j * d.L
                                  : reinterpret_cast<const float2 *>(nparams) + ((size_t)row * d.J + j) * d.L;
            }
            float ab[DCMAX][V], mn1[V], mn2[V];
            uint32_t neg[V];
#pragma unroll
            for (int v = 0; v < V; ++v) mn1[v] = mn2[v] = INFINITY, neg[v] = 0u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
#pragma unroll
                for (int v = 0; v < V; ++v) ab[l][v] = INFINITY;
                if (REG || l < LB) {
                    const int o = __shfl_sync(0xffffffffu, myoff, l);
                    if (REG || o >= 0) {
                        float x[V];
                        Lane<V>::unpack(S[l * 32 + lane], x);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const float a = fabsf(x[v]);
                            ab[l][v] = a;
                            neg[v] |= (x[v] < 0.0f ? 1u : 0u) << l;
                            mn2[v] = fminf(mn2[v], fmaxf(mn1[v], a));
                            mn1[v] = fminf(mn1[v], a);
                        }
                    }
                }
            }
            uint32_t par_all[V];
#pragma unroll
            for (int v = 0; v < V; ++v) par_all[v] = __popc(neg[v]) & 1u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const int o = __shfl_sync(0xffffffffu, myoff, l);
                if (!REG && o < 0) continue;
                float out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float2 wo = prm_smem ? prm[v][l] : __ldg(prm[v] + l);
                    const float m = ab[l][v] == mn1[v] ? mn2[v] : mn1[v];
                    const float mag = fminf(fmaxf(fmaf(wo.x, m, -wo.y), 0.0f), clip);
                    out[v] = (par_all[v] ^ ((neg[v] >> l) & 1u)) ? -mag : mag;
                    if (fr[v]) out[v] = 0.0f;
                }
                if (lane_on) gmsg[(size_t)o * 32] = Lane<V>::pack(out);
            }
        } else {
            // min-sum, 4 frames per lane word (V == 4)
            uint32_t ab[DCMAX], sg[DCMAX];
            uint32_t min1 = 0x7f7f7f7fu, min2 = 0x7f7f7f7fu, sgn = 0u;
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                ab[l] = 0u;
                sg[l] = 0u;
                if (REG || l < LB) {
                    const int o = __shfl_sync(0xffffffffu, myoff, l);
                    if (REG || o >= 0) {
                        const uint32_t x = S[l * 32 + lane];
                        const uint32_t av = __vabsss4(x);
                        sg[l] = x & 0x80808080u;
                        ab[l] = av;
                        sgn ^= sg[l];
                        min2 = __vminu4(min2, __vmaxu4(min1, av));
                        min1 = __vminu4(min1, av);
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < DCMAX; ++l) {
                const int o = __shfl_sync(0xffffffffu, myoff, l);
                if (!REG && o < 0) continue;
                const uint32_t eq = __vcmpeq4(ab[l], min1);
                const uint32_t mag = (min2 & eq) | (min1 & ~eq);
                const uint32_t sneg = ((sgn ^ sg[l]) >> 7) & 0x01010101u;
                if (lane_on) gmsg[(size_t)o * 32] = __vadd4(mag ^ (sneg * 0xffu), sneg) & ~frmask;
            }
        }
        __syncwarp();
        slot = (slot + 1) % kCnStages;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// variable pass: eqs. (bpvs), (bpd), (hrddcs) on kNV consecutive variables.
// REG: every block of the column is present and J == JMAX.
// ---------------------------------------------------------------------------
template <int JMAX, int V, bool STOP, bool MS>
struct VnStage {
    static constexpr int MUW = MS ? 32 : 32 * V;     // channel-LLR words per variable
    static constexpr int MU = 0;
    static constexpr int AL = kNV * MUW;             // [i][j][32] edge packages
    static constexpr int HW = AL + kNV * JMAX * 32;  // old hard words [i][V]
    static constexpr int FL = HW + kNV * V;          // done[V], then unsat[V] (continuous simulation: retire[V])
    static constexpr int NFL = 2 * V;
    static constexpr int WORDS = (FL + NFL + 3) & ~3;
};

// EVEN: N is a multiple of kNV (every item has kNV variables)
// SPARSE: a general code (each variable's edges from index tables)
template <int JMAX, int V, bool STOP, bool POST, bool XF, bool MS, bool REG, bool REFILL = false, bool EVEN = false,
          bool SPARSE = false>
__global__ void __launch_bounds__(kWarps * 32)
vn_pipe_kernel(const QcDesc d, uint32_t *__restrict__ msg, uint32_t *__restrict__ mu, uint32_t *__restrict__ hw,
               uint32_t *__restrict__ flags, float *__restrict__ post, int32_t *__restrict__ iters,
               const int *__restrict__ act, float clip, float lsb, int it, int par, RefillArgs rf, SparseTab tab) {
    static_assert(!(SPARSE && (REG || REFILL)), "general codes: irregular columns, batch decoding");
    using St = VnStage<JMAX, V, STOP, MS>;
    constexpr int W = 32 * V;
    static_assert(kNV == 4, "items of 4 variables: 16-byte channel rows, 4-byte lane words");
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_sh[kMaxJ * kMaxL], s_eo[kMaxJ * kMaxL];
    for (int i = threadIdx.x; i < d.J * d.L; i += blockDim.x) {
        s_sh[i] = d.shift[i];
        s_eo[i] = d.eoff[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kVnStages * St::WORDS;
    const int G = (d.N + kNV - 1) / kNV;
    const int total = act[0] * G;  // work items (package, group of kNV variables)
    const int *list = act + 1;
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;
    constexpr int MU_SEGS = St::MUW / 32;

    // starts the copies of item itm into ring slot `slot`; returns this lane's edge offset
    // (lane t < kNV * JMAX: edge (variable t / JMAX, block row t % JMAX), -1 if absent)
    auto issue = [&](int itm, int slot) -> int {
        int mine = -1;
        if (itm < total) {
            const int a = (int)fdiv((uint32_t)itm, d.divG);
            const int g = itm - a * G;
            const int pk = __ldg(list + a);
            uint32_t *dst = ring + slot * St::WORDS;
            const uint32_t *gmsg = msg + (size_t)pk * d.E * 32;
            const uint32_t *gmu = mu + (size_t)pk * d.N * St::MUW;
            const int n0 = g * kNV;
            const int l0 = (int)fdiv((uint32_t)n0, d.divP), k0 = n0 - l0 * d.p;
            const int grp = lane >> 3, sub = lane & 7;
            if (REFILL) {
                // continuous simulation: frame-major channel LLRs [P][W][N4] (rows padded to a
                // multiple of 4): each lane copies its V frames' kNV values, [lane][v][kNV] in the ring
                const size_t N4 = (size_t)((d.N + 3) & ~3);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const size_t row = (size_t)pk * W + lane * V + v;
                    if constexpr (MS)
                        cp_async4(dst + St::MU + lane * 4 + v,
                                  reinterpret_cast<const uint8_t *>(rf.mu) + row * N4 + n0);
                    else
                        cp_async16(dst + St::MU + (lane * V + v) * 4,
                                   reinterpret_cast<const float *>(rf.mu) + row * N4 + n0);
                }
            } else {
                // channel LLRs: kNV * MU_SEGS segments of 32 words, one per group of 8 lanes and pass
#pragma unroll
                for (int s0 = 0; s0 < kNV * MU_SEGS; s0 += 4) {
                    const int s = s0 + grp;
                    const int i = s / MU_SEGS, h = s - i * MU_SEGS;
                    const int n = n0 + i;
                    if ((kNV * MU_SEGS) % 4 == 0 || s < kNV * MU_SEGS)
                        if (EVEN || n < d.N)
                            cp_async16(dst + St::MU + i * St::MUW + h * 32 + sub * 4,
                                       gmu + (size_t)n * St::MUW + h * 32 + sub * 4);
                }
            }
            if constexpr (SPARSE) {
                // each variable's edges from the tables: lane t < kNV * JMAX looks up edge t % JMAX
                // of variable t / JMAX; the lane groups copy the packages
                if (lane < kNV * JMAX) {
                    const int i = lane / JMAX, jj = lane - i * JMAX;
                    const int n = n0 + i;
                    if (n < d.N) {
                        const int c0 = __ldg(tab.cptr + n), deg = __ldg(tab.cptr + n + 1) - c0;
                        if (jj < deg) mine = __ldg(tab.cedge + c0 + jj);
                    }
                }
#pragma unroll
                for (int t0 = 0; t0 < kNV * JMAX; t0 += 4) {
                    const int e = __shfl_sync(0xffffffffu, mine, t0 + grp);
                    if (e >= 0) cp_async16(dst + St::AL + (t0 + grp) * 32 + sub * 4, gmsg + (size_t)e * 32 + sub * 4);
                }
            } else {
                // edge packages: kNV * JMAX of them; lane t computes edge t's offset once and the
                // copies take it by shuffle
                if (lane < kNV * JMAX) {
                    const int i = lane / JMAX, jj = lane - i * JMAX;
                    int l = l0, k = k0 + i;
                    if (k >= d.p) k -= d.p, ++l;
                    if ((EVEN || n0 + i < d.N) && (REG || (jj < d.J && s_sh[jj * d.L + l] >= 0)))
                        mine = s_eo[jj * d.L + l] + k;
                }
#pragma unroll
                for (int t0 = 0; t0 < kNV * JMAX; t0 += 4) {
                    const int t = t0 + grp;
                    const int e = __shfl_sync(0xffffffffu, mine, t & 31);
                    if (((kNV * JMAX) % 4 == 0 || t < kNV * JMAX) && ((REG && EVEN) || e >= 0))
                        cp_async16(dst + St::AL + t * 32 + sub * 4, gmsg + (size_t)e * 32 + sub * 4);
                }
            }
            if (lane < kNV * V) {
                const int i = lane / V, v = lane - i * V;
                const int n = n0 + i;
                if (EVEN || n < d.N) cp_async4(dst + St::HW + lane, hw + ((size_t)pk * d.N + n) * V + v);
            } else if (lane >= 32 - St::NFL) {
                const int q = lane - (32 - St::NFL);
                if (REFILL) {
                    // done[V] (slots without a running frame), retire[V]
                    if (q < V) cp_async4(dst + St::FL + q, flags + (size_t)pk * 5 * V + q);
                    else cp_async4(dst + St::FL + q, rf.sflags + (size_t)pk * 2 * V + (q - V));
                } else {
                    // done[V], unsat[par][V]
                    const int off = q < V ? q : (1 + par) * V + (q - V);
                    cp_async4(dst + St::FL + q, flags + (size_t)pk * 5 * V + off);
                }
            }
        }
        cp_async_commit();
        return mine;
    };

    int offr[kVnStages];
#pragma unroll
    for (int s = 0; s < kVnStages - 1; ++s) offr[s] = issue(item + s * GW, s);
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kVnStages - 1] = issue(item + (kVnStages - 1) * GW, (slot + kVnStages - 1) % kVnStages);
        cp_async_wait<kVnStages - 1>();
        __syncwarp();
        const uint32_t *S = ring + slot * St::WORDS;
        const int myoff = offr[0];
#pragma unroll
        for (int s = 0; s < kVnStages - 1; ++s) offr[s] = offr[s + 1];
        const int a = (int)fdiv((uint32_t)item, d.divG);
        const int g = item - a * G;
        const int pk = __ldg(list + a);
        uint32_t *gmsg = msg + (size_t)pk * d.E * 32 + lane;
        // frames stopped so far, and the ones whose last decisions satisfied every check
        uint32_t frozen[V], retire[V];
        bool lane_on = false;
        if (REFILL) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                retire[v] = S[St::FL + V + v];
                frozen[v] = S[St::FL + v];
                lane_on |= ((~frozen[v]) >> lane) & 1u;
            }
        }
#pragma unroll
        for (int v = 0; v < V && !REFILL; ++v) {
            uint32_t dn = S[St::FL + v];
            if (STOP) {
                const uint32_t newly = ~dn & ~S[St::FL + V + v];
                if (g == 0 && lane == 0) {
                    uint32_t *F = flags + (size_t)pk * 5 * V;
                    if (newly) {
                        F[v] = dn | newly;
                        for (uint32_t b = newly; b; b &= b - 1) {
                            const int ln = __ffs(b) - 1;
                            iters[(size_t)pk * W + ln * V + v] = it - 1;
                        }
                    }
                    F[(1 + (par ^ 1)) * V + v] = 0u;  // cleared for the next check pass
                }
                dn |= newly;
            }
            frozen[v] = dn;
            lane_on |= ((~dn) >> lane) & 1u;
        }
        const int n0 = g * kNV;
        if (REFILL) {
            // wrong bits of the frames that retired this step: their last decisions are the staged
            // hard words (a new frame in the same slot writes its first decisions below)
            bool any_retire = false;
#pragma unroll
            for (int v = 0; v < V; ++v) any_retire |= retire[v] != 0u;
            if (any_retire && rf.errs != nullptr) {  // NULL: counted against sent codewords elsewhere
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (!((retire[v] >> lane) & 1u)) continue;
                    int cnt = 0;
#pragma unroll
                    for (int i = 0; i < kNV; ++i)
                        if (EVEN || n0 + i < d.N) cnt += (S[St::HW + i * V + v] >> lane) & 1u;
                    if (cnt) atomicAdd(rf.errs + (size_t)pk * W + lane * V + v, cnt);
                }
            }
        }
        // continuous simulation: this lane's channel values, frame-major in the ring
        float mr[MS ? 1 : V][kNV];
        uint32_t qr[kNV];
        if constexpr (REFILL) {
            if constexpr (MS) {
                // words v: the kNV bytes of frame v; transpose to words i: frames 0..3 of variable i
                const uint4 wv = *reinterpret_cast<const uint4 *>(S + St::MU + lane * 4);
                const uint32_t a01 = __byte_perm(wv.x, wv.y, 0x5140), a23 = __byte_perm(wv.z, wv.w, 0x5140);
                const uint32_t b01 = __byte_perm(wv.x, wv.y, 0x7362), b23 = __byte_perm(wv.z, wv.w, 0x7362);
                qr[0] = __byte_perm(a01, a23, 0x5410);
                qr[1] = __byte_perm(a01, a23, 0x7632);
                qr[2] = __byte_perm(b01, b23, 0x5410);
                qr[3] = __byte_perm(b01, b23, 0x7632);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float4 f = *reinterpret_cast<const float4 *>(S + St::MU + (lane * V + v) * 4);
                    mr[v][0] = f.x, mr[v][1] = f.y, mr[v][2] = f.z, mr[v][3] = f.w;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kNV; ++i) {
            const int n = n0 + i;
            if (!EVEN && n >= d.N) break;  // warp-uniform
            // the item's edge offsets (-1: absent), warp-uniform
            int eo[JMAX];
#pragma unroll
            for (int jj = 0; jj < JMAX; ++jj) eo[jj] = __shfl_sync(0xffffffffu, myoff, i * JMAX + jj);
            uint32_t outb[V];
            if constexpr (!MS) {
                float m[V], aj[JMAX][V], tot[V];
                const float *mf = reinterpret_cast<const float *>(S + St::MU + i * St::MUW) + lane * V;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    m[v] = REFILL ? mr[v][i] : mf[v];
                    tot[v] = m[v];
                }
#pragma unroll
                for (int jj = 0; jj < JMAX; ++jj) {
                    const bool on = REG || eo[jj] >= 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) aj[jj][v] = 0.0f;
                    if (on) {
                        Lane<V>::unpack(S[St::AL + (i * JMAX + jj) * 32 + lane], aj[jj]);
#pragma unroll
                        for (int v = 0; v < V; ++v) tot[v] += aj[jj][v];
                    }
                }
                // extrinsic sums beta = mu + the other edges' alpha
                float bs[JMAX][V];
#pragma unroll
                for (int jj = 0; jj < JMAX; ++jj)
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        float s = m[v];
#pragma unroll
                        for (int j2 = 0; j2 < JMAX; ++j2)
                            if (j2 != jj) s += aj[j2][v];
                        bs[jj][v] = s;
                    }
                if constexpr (XF) {
                    // the check pass sums phi(|beta|): evaluate it here, from the unrounded beta
                    // (|clip(s)| = min(|s|, clip)), keep beta's sign; packed pairs as in the check pass
                    float ph[JMAX][V];
                    if constexpr (V == 2) {
#pragma unroll
                        for (int jj = 0; jj < JMAX; ++jj)
                            phi_fin2(fminf(fabsf(bs[jj][0]), clip), fminf(fabsf(bs[jj][1]), clip), ph[jj][0],
                                     ph[jj][1]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj + 1 < JMAX; jj += 2)
                            phi_fin2(fminf(fabsf(bs[jj][0]), clip), fminf(fabsf(bs[jj + 1][0]), clip), ph[jj][0],
                                     ph[jj + 1][0]);
                        if (JMAX % 2) ph[JMAX - 1][0] = phi_fin(fminf(fabsf(bs[JMAX - 1][0]), clip));
                    }
#pragma unroll
                    for (int jj = 0; jj < JMAX; ++jj)
#pragma unroll
                        for (int v = 0; v < V; ++v) bs[jj][v] = with_sign_of(ph[jj][v] * XfScale<V>::store, bs[jj][v]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < JMAX; ++jj)
#pragma unroll
                        for (int v = 0; v < V; ++v) bs[jj][v] = clipf(bs[jj][v], clip);
                }
#pragma unroll
                for (int jj = 0; jj < JMAX; ++jj) {
                    if (!REG && eo[jj] < 0) continue;  // warp-uniform
                    if (lane_on) gmsg[(size_t)eo[jj] * 32] = Lane<V>::pack(bs[jj]);
                }
                float pst[V];
#pragma unroll
                for (int v = 0; v < V; ++v) pst[v] = clipf(tot[v], clip);
                if (POST && lane_on) {
                    float *dst = post + ((size_t)pk * d.N + n) * W + lane * V;
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (!((frozen[v] >> lane) & 1u)) dst[v] = pst[v];
                }
#pragma unroll
                for (int v = 0; v < V; ++v) outb[v] = __ballot_sync(0xffffffffu, pst[v] < 0.0f);
            } else {
                const uint32_t qw = REFILL ? qr[i] : S[St::MU + i * St::MUW + lane];
                uint32_t aw[JMAX];
                int tot[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) tot[v] = sbyte(qw, v);
#pragma unroll
                for (int jj = 0; jj < JMAX; ++jj) {
                    const bool on = REG || eo[jj] >= 0;
                    aw[jj] = on ? S[St::AL + (i * JMAX + jj) * 32 + lane] : 0u;
#pragma unroll
                    for (int v = 0; v < 4; ++v) tot[v] += sbyte(aw[jj], v);
                }
                if (lane_on) {
#pragma unroll
                    for (int jj = 0; jj < JMAX; ++jj) {
                        if (!REG && eo[jj] < 0) continue;
                        uint32_t o = 0u;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            int b = tot[v] - sbyte(aw[jj], v);
                            b = b > 127 ? 127 : (b < -127 ? -127 : b);
                            o |= ((uint32_t)(uint8_t)(int8_t)b) << (8 * v);
                        }
                        gmsg[(size_t)eo[jj] * 32] = o;
                    }
                }
                if (POST && lane_on) {
                    float *dst = post + ((size_t)pk * d.N + n) * W + lane * V;
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (!((frozen[v] >> lane) & 1u)) dst[v] = (float)tot[v] * lsb;
                }
#pragma unroll
                for (int v = 0; v < V; ++v) outb[v] = __ballot_sync(0xffffffffu, tot[v] < 0);
            }
            if (lane == 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t old = S[St::HW + i * V + v];
                    hw[((size_t)pk * d.N + n) * V + v] = (outb[v] & ~frozen[v]) | (old & frozen[v]);
                }
            }
        }
        __syncwarp();
        slot = (slot + 1) % kVnStages;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// list of packages with at least one frame still running: act[0] = count,
// act[1..] = package indices (one block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) compact_kernel(const uint32_t *__restrict__ flags,
                                                       int P, int V,
                                                       int *__restrict__ act) {
    __shared__ int wsum[32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p0 = 0; p0 < P; p0 += blockDim.x) {
        const int pk = p0 + threadIdx.x;
        bool on = false;
        if (pk < P)
            for (int v = 0; v < V; ++v) on |= ~flags[(size_t)pk * 5 * V + v] != 0u;
        const uint32_t bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += wsum[w];
            all += wsum[w];
        }
        const int base = s_base;
        if (on) act[1 + base + before + __popc(bal & ((1u << lane) - 1u))] = pk;
        __syncthreads();
        if (threadIdx.x == 0) s_base = base + all;
        __syncthreads();
    }
    if (threadIdx.x == 0) act[0] = s_base;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <int DCMAX, int V, bool XF, int MODE, bool REG>
static void launch_cn_pipe(ldpc_code c, const ldpc_decode_opts &o, int it, const uint32_t *fresh, const int *ages,
                           cudaStream_t s) {
    auto k = cn_pipe_kernel<DCMAX, V, XF, MODE, REG>;
    size_t smem = (size_t)kWarps * kCnStages * (CnStage<DCMAX>::WORDS + (MODE == kModeNOMS ? 32 * V : 0)) * 4;
    if (MODE == kModeNOMS && ages) {
        const int PS = ((c->d.J * c->d.L + 14) / 16) * 16 + 1;
        const size_t tb = (size_t)o.max_iter * PS * 8;
        if (tb <= (size_t)kNomsSmemTable) smem += tb;
    }
    const int blocks = persistent_blocks(k, smem);
    // per-frame rows (ages): the whole table; else this iteration's row
    const float *np = !o.noms_params ? nullptr
                      : ages ? o.noms_params
                             : o.noms_params + (size_t)(it - 1) * c->d.J * c->d.L * 2;
    k<<<blocks, kWarps * 32, smem, s>>>(c->d, (uint32_t *)c->ws.msg, c->ws.flags, fresh, c->ws.act, o.clip, np,
                                        ages, o.max_iter, SparseTab());
}

template <int DCMAX, bool REG>
static void cn_pipe_dispatch(ldpc_code c, const ldpc_decode_opts &o, int it, const uint32_t *fresh, const int *ages,
                             cudaStream_t s) {
    if (o.algo == LDPC_ALGO_MS) launch_cn_pipe<DCMAX, 4, false, kModeMS, REG>(c, o, it, fresh, ages, s);
    else if (o.algo == LDPC_ALGO_NOMS) {
        if (o.msg == LDPC_MSG_F16) launch_cn_pipe<DCMAX, 2, false, kModeNOMS, REG>(c, o, it, fresh, ages, s);
        else launch_cn_pipe<DCMAX, 1, false, kModeNOMS, REG>(c, o, it, fresh, ages, s);
    } else if (o.msg == LDPC_MSG_F16) {
        launch_cn_pipe<DCMAX, 2, true, kModeSP, REG>(c, o, it, fresh, ages, s);
    } else {
        launch_cn_pipe<DCMAX, 1, true, kModeSP, REG>(c, o, it, fresh, ages, s);
    }
}

// a regular code whose row degree is exactly one of the compiled degrees
static bool regular_rows(const QcDesc &d, int dcmax) {
    if (d.L != dcmax) return false;
    for (int i = 0; i < d.J * d.L; ++i)
        if (d.shift[i] < 0) return false;
    return true;
}

ldpc_status qc_cn_pipe(ldpc_code c, const ldpc_decode_opts &o, int it, cudaStream_t s, const uint32_t *fresh,
                       const int *ages) {
    const QcDesc &d = c->d;
    if (regular_rows(d, 24)) cn_pipe_dispatch<24, true>(c, o, it, fresh, ages, s);
    else if (d.L <= 8) cn_pipe_dispatch<8, false>(c, o, it, fresh, ages, s);
    else if (d.L <= 16) cn_pipe_dispatch<16, false>(c, o, it, fresh, ages, s);
    else if (d.L <= 24) cn_pipe_dispatch<24, false>(c, o, it, fresh, ages, s);
    else cn_pipe_dispatch<32, false>(c, o, it, fresh, ages, s);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

template <int JMAX, int V, bool STOP, bool POST, bool XF, bool MS, bool REG>
static void launch_vn_pipe(ldpc_code c, const ldpc_decode_opts &o, int it, int par, cudaStream_t s) {
    auto k = (REG && c->d.N % kNV == 0) ? vn_pipe_kernel<JMAX, V, STOP, POST, XF, MS, REG, false, REG>
                                        : vn_pipe_kernel<JMAX, V, STOP, POST, XF, MS, REG, false, false>;
    const size_t smem = (size_t)kWarps * kVnStages * VnStage<JMAX, V, STOP, MS>::WORDS * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(c->d, (uint32_t *)c->ws.msg, (uint32_t *)c->ws.mu, c->ws.hw, c->ws.flags,
                                        c->ws.post, c->ws.iters, c->ws.act, o.clip, ldexpf(1.0f, -o.frac_bits), it,
                                        par, RefillArgs{}, SparseTab());
}

template <int JMAX, bool STOP, bool POST, bool REG>
static void vn_pipe_dispatch(ldpc_code c, const ldpc_decode_opts &o, int it, int par, cudaStream_t s) {
    // sum-product stores transformed messages; learned min-sum (NOMS) needs beta itself
    if (o.algo == LDPC_ALGO_MS) launch_vn_pipe<JMAX, 4, STOP, POST, false, true, REG>(c, o, it, par, s);
    else if (o.algo == LDPC_ALGO_NOMS && o.msg == LDPC_MSG_F16)
        launch_vn_pipe<JMAX, 2, STOP, POST, false, false, REG>(c, o, it, par, s);
    else if (o.algo == LDPC_ALGO_NOMS) launch_vn_pipe<JMAX, 1, STOP, POST, false, false, REG>(c, o, it, par, s);
    else if (o.msg == LDPC_MSG_F16) launch_vn_pipe<JMAX, 2, STOP, POST, true, false, REG>(c, o, it, par, s);
    else launch_vn_pipe<JMAX, 1, STOP, POST, true, false, REG>(c, o, it, par, s);
}

template <int JMAX, bool REG>
static void vn_pipe_dispatch2(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                              cudaStream_t s) {
    if (stop) {
        if (post) vn_pipe_dispatch<JMAX, true, true, REG>(c, o, it, par, s);
        else vn_pipe_dispatch<JMAX, true, false, REG>(c, o, it, par, s);
    } else {
        if (post) vn_pipe_dispatch<JMAX, false, true, REG>(c, o, it, par, s);
        else vn_pipe_dispatch<JMAX, false, false, REG>(c, o, it, par, s);
    }
}

ldpc_status qc_vn_pipe(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                       cudaStream_t s) {
    const QcDesc &d = c->d;
    bool full = true;
    for (int i = 0; i < d.J * d.L; ++i) full &= d.shift[i] >= 0;
    if (full && d.J == 4) vn_pipe_dispatch2<4, true>(c, o, stop, post, it, par, s);
    else if (full && d.J == 3) vn_pipe_dispatch2<3, true>(c, o, stop, post, it, par, s);
    else if (d.J <= 4) vn_pipe_dispatch2<4, false>(c, o, stop, post, it, par, s);
    else vn_pipe_dispatch2<8, false>(c, o, stop, post, it, par, s);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status qc_compact(ldpc_code c, int P, int V, cudaStream_t s) {
    compact_kernel<<<1, 1024, 0, s>>>(c->ws.flags, P, V, c->ws.act);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

namespace ldpc {

// variable pass of the continuous simulation: no early-stop bookkeeping (the
// retire kernel owns the flag words), no posteriors
template <int JMAX, int V, bool XF, bool MS, bool REG>
static void launch_vn_refill(ldpc_code c, const ldpc_decode_opts &o, const RefillArgs &rf, cudaStream_t s) {
    auto k = (REG && c->d.N % kNV == 0) ? vn_pipe_kernel<JMAX, V, false, false, XF, MS, REG, true, REG>
                                        : vn_pipe_kernel<JMAX, V, false, false, XF, MS, REG, true, false>;
    const size_t smem = (size_t)kWarps * kVnStages * VnStage<JMAX, V, false, MS>::WORDS * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(c->d, (uint32_t *)c->ws.msg, (uint32_t *)c->ws.mu, c->ws.hw, c->ws.flags,
                                        nullptr, nullptr, c->ws.act, o.clip, ldexpf(1.0f, -o.frac_bits), 0, 0, rf,
                                        SparseTab());
}

template <int JMAX, bool REG>
static void vn_refill_dispatch(ldpc_code c, const ldpc_decode_opts &o, const RefillArgs &rf, cudaStream_t s) {
    if (o.algo == LDPC_ALGO_MS) launch_vn_refill<JMAX, 4, false, true, REG>(c, o, rf, s);
    else if (o.algo == LDPC_ALGO_NOMS && o.msg == LDPC_MSG_F16) launch_vn_refill<JMAX, 2, false, false, REG>(c, o, rf, s);
    else if (o.algo == LDPC_ALGO_NOMS) launch_vn_refill<JMAX, 1, false, false, REG>(c, o, rf, s);
    else if (o.msg == LDPC_MSG_F16) launch_vn_refill<JMAX, 2, true, false, REG>(c, o, rf, s);
    else launch_vn_refill<JMAX, 1, true, false, REG>(c, o, rf, s);
}

ldpc_status qc_vn_refill(ldpc_code c, const ldpc_decode_opts &o, const RefillArgs &rf, cudaStream_t s) {
    const QcDesc &d = c->d;
    bool full = true;
    for (int i = 0; i < d.J * d.L; ++i) full &= d.shift[i] >= 0;
    if (full && d.J == 4) vn_refill_dispatch<4, true>(c, o, rf, s);
    else if (full && d.J == 3) vn_refill_dispatch<3, true>(c, o, rf, s);
    else if (d.J <= 4) vn_refill_dispatch<4, false>(c, o, rf, s);
    else vn_refill_dispatch<8, false>(c, o, rf, s);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

namespace ldpc {

// ---------------------------------------------------------------------------
// general (index-table) codes: the same passes with table-driven copy stages
// ---------------------------------------------------------------------------
template <int DCMAX, int V, bool XF, int MODE>
static void launch_cn_sparse(ldpc_code c, const ldpc_decode_opts &o, cudaStream_t s) {
    auto k = cn_pipe_kernel<DCMAX, V, XF, MODE, false, true>;
    const size_t smem = (size_t)kWarps * kCnStages * CnStage<DCMAX>::WORDS * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(c->d, (uint32_t *)c->ws.msg, c->ws.flags, nullptr, c->ws.act, o.clip,
                                        nullptr, nullptr, 0, c->sp);
}

template <int DCMAX>
static void cn_sparse_dispatch(ldpc_code c, const ldpc_decode_opts &o, cudaStream_t s) {
    if (o.algo == LDPC_ALGO_MS) launch_cn_sparse<DCMAX, 4, false, kModeMS>(c, o, s);
    else if (o.msg == LDPC_MSG_F16) launch_cn_sparse<DCMAX, 2, true, kModeSP>(c, o, s);
    else launch_cn_sparse<DCMAX, 1, true, kModeSP>(c, o, s);
}

ldpc_status qc_cn_pipe_sparse(ldpc_code c, const ldpc_decode_opts &o, cudaStream_t s) {
    const int dc = c->sp.dc_max;
    if (dc <= 8) cn_sparse_dispatch<8>(c, o, s);
    else if (dc <= 16) cn_sparse_dispatch<16>(c, o, s);
    else if (dc <= 24) cn_sparse_dispatch<24>(c, o, s);
    else cn_sparse_dispatch<32>(c, o, s);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

template <int JMAX, int V, bool STOP, bool POST, bool XF, bool MS>
static void launch_vn_sparse(ldpc_code c, const ldpc_decode_opts &o, int it, int par, cudaStream_t s) {
    auto k = vn_pipe_kernel<JMAX, V, STOP, POST, XF, MS, false, false, false, true>;
    const size_t smem = (size_t)kWarps * kVnStages * VnStage<JMAX, V, STOP, MS>::WORDS * 4;
    const int blocks = persistent_blocks(k, smem);
    k<<<blocks, kWarps * 32, smem, s>>>(c->d, (uint32_t *)c->ws.msg, (uint32_t *)c->ws.mu, c->ws.hw, c->ws.flags,
                                        c->ws.post, c->ws.iters, c->ws.act, o.clip, ldexpf(1.0f, -o.frac_bits), it,
                                        par, RefillArgs{}, c->sp);
}

template <int JMAX, bool STOP, bool POST>
static void vn_sparse_dispatch(ldpc_code c, const ldpc_decode_opts &o, int it, int par, cudaStream_t s) {
    if (o.algo == LDPC_ALGO_MS) launch_vn_sparse<JMAX, 4, STOP, POST, false, true>(c, o, it, par, s);
    else if (o.msg == LDPC_MSG_F16) launch_vn_sparse<JMAX, 2, STOP, POST, true, false>(c, o, it, par, s);
    else launch_vn_sparse<JMAX, 1, STOP, POST, true, false>(c, o, it, par, s);
}

template <int JMAX>
static void vn_sparse_dispatch2(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                                cudaStream_t s) {
    if (stop) {
        if (post) vn_sparse_dispatch<JMAX, true, true>(c, o, it, par, s);
        else vn_sparse_dispatch<JMAX, true, false>(c, o, it, par, s);
    } else {
        if (post) vn_sparse_dispatch<JMAX, false, true>(c, o, it, par, s);
        else vn_sparse_dispatch<JMAX, false, false>(c, o, it, par, s);
    }
}

ldpc_status qc_vn_pipe_sparse(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                              cudaStream_t s) {
    if (c->sp.dv_max <= 4) vn_sparse_dispatch2<4>(c, o, stop, post, it, par, s);
    else vn_sparse_dispatch2<8>(c, o, stop, post, it, par, s);
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

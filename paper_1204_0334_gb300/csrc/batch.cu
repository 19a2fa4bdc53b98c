// Heterogeneous batches: many QC codes, each with its own number of frames,
// decoded together (Algorithm 1 for every code, one shared iteration loop).
//
// Every code keeps the single-code layout (packages of W = 32*V frames,
// msg [P][E][32], mu [P][N][W], hw [P][N][V], flags) inside one workspace.
// Work is a list of tiles (code, package, first row or variable group, count):
// after every variable pass a compaction kernel lists the tiles of the
// packages that still have a running frame, across all codes, so one
// persistent check-pass launch and one variable-pass launch per iteration
// serve the whole batch and converged packages of any code drop out
// (active-frame compaction at package granularity).  Warps stage each item's
// 128-byte edge packages with cp.async into a shared-memory ring, as the
// single-code passes do; codes are read from a device table (their shift and
// edge-offset tables sit in global memory, cached in L1).
//
// The iteration loop (check pass, variable pass, compaction) is captured once
// into a CUDA graph and replayed by later calls.  The first call tunes the tile
// sizes (rows per check-pass tile, variable groups per variable-pass tile) by
// timing a few iterations of each candidate on the call's own frames.
#include "qc_device.cuh"

#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <memory>
#include <vector>

namespace ldpc {

struct BCode {
    int J, L, p, N, M, E, P, gamma, tab;
    FastDiv dp;                           // n / p by multiply-high
    long long msg, mu, hw, flags, iters;  // offsets (words / ints) into the shared regions
    long long map;                        // offset of the code's compaction map (ints)
};

struct BTile {
    int code, pk, start, count;
};

static_assert(sizeof(BTile) == 16, "one 16-byte load per tile");
// tile i of a list the pass only reads (the list is 16-byte aligned)
__device__ __forceinline__ BTile b_tile(const BTile *tiles, int i) {
    const int4 t = __ldg(reinterpret_cast<const int4 *>(tiles) + i);
    return BTile{t.x, t.y, t.z, t.w};
}

constexpr int kBStages = 3;
constexpr int kBDC = 24;  // largest row degree of a batch
constexpr int kBJ = 4;    // largest column degree of a batch
constexpr int kBNV = 4;   // variables per variable-pass item

__device__ __forceinline__ uint32_t b_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void b_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(b_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void b_cp4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(b_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void b_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void b_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int V, bool FIRST, bool MS>
struct BCnStage {
    static constexpr int MUW = MS ? 32 : 32 * V;     // words of one channel-LLR package
    static constexpr int SEGW = FIRST ? MUW : 32;    // words per edge in the stage
    static constexpr int SEG = kBDC * SEGW;
    static constexpr int FL = SEG;
    static constexpr int WORDS = (FL + V + 3) & ~3;
};

// ---------------------------------------------------------------------------
// check pass over all codes (FIRST: beta = mu)
// ---------------------------------------------------------------------------
template <int V, bool XF, bool MS, bool FIRST>
__global__ void __launch_bounds__(kWarps * 32, 2)  // two blocks of eight warps per SM
bcn_kernel(const BCode *__restrict__ codes, const int *__restrict__ shtab, const int *__restrict__ eotab,
           uint32_t *__restrict__ msg, const uint32_t *__restrict__ mu, const uint32_t *__restrict__ flags,
           const int *__restrict__ tcount, const BTile *__restrict__ tiles, int TR, float clip) {
    using St = BCnStage<V, FIRST, MS>;
    const int sTR = __ffs(TR) - 1;  // TR is a power of two
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kBStages * St::WORDS;
    const int total = *tcount * TR;
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;

    // starts the copies of item it; returns this lane's edge offset (lane l < kBDC: edge l of
    // the row in 32-word packages, -1 if absent)
    // the message base (words) of each staged item, -1 for an empty item: the compute phase
    // needs nothing else from the tile and code tables
    long long gbase[kBStages];
    long long base_out = -1;  // the base of the item issue() staged last
    // the row degree slot bound (edge slots >= it are absent) of each staged item
    int gdeg[kBStages];
    int deg_out = 0;
    // the tile of the next item this warp stages, loaded one item ahead (items are staged in
    // order it, it + GW, ...), so that staging waits on the code tables only
    BTile tl_next = item < total ? b_tile(tiles, item >> sTR) : BTile{0, 0, 0, 0};
    auto issue = [&](int it, int slot) -> int {
        int mine = -1;
        long long base = -1;
        int deg = 0;
        const BTile tl = tl_next;
        if (it + GW < total) tl_next = b_tile(tiles, (it + GW) >> sTR);
        if (it < total) {
            const int ri = it & (TR - 1);
            if (ri < tl.count) {
                const BCode C = codes[tl.code];
                const int m = tl.start + ri;
                const int j = (int)fdiv((uint32_t)m, C.dp), r = m - j * C.p;
                base = C.msg + (long long)tl.pk * C.E * 32;
                deg = C.L;
                uint32_t *dst = ring + slot * St::WORDS;
                const uint32_t *gsrc = FIRST ? mu + C.mu + (size_t)tl.pk * C.N * St::MUW
                                             : msg + C.msg + (size_t)tl.pk * C.E * 32;
                const int g = lane >> 3, sub = lane & 7;
                // lane l looks up edge l of the row once (its offset, and its variable for FIRST);
                // the copies take them by shuffle
                int my_n = 0;
                if (lane < kBDC && lane < C.L) {
                    const int sh = __ldg(shtab + C.tab + j * C.L + lane);
                    if (sh >= 0) {
                        int k = r + sh;
                        if (k >= C.p) k -= C.p;
                        mine = __ldg(eotab + C.tab + j * C.L + lane) + k;
                        my_n = lane * C.p + k;
                    }
                }
#pragma unroll
                for (int q = 0; q < kBDC / 4; ++q) {
                    const int l = 4 * q + g;
                    const int o = __shfl_sync(0xffffffffu, mine, l);
                    if (FIRST) {
                        const int n = __shfl_sync(0xffffffffu, my_n, l);
                        if (o >= 0) {
#pragma unroll
                            for (int h = 0; h < St::MUW / 32; ++h)
                                b_cp16(dst + l * St::SEGW + h * 32 + sub * 4, gsrc + (size_t)n * St::MUW + h * 32 + sub * 4);
                        }
                    } else if (o >= 0) {
                        b_cp16(dst + l * 32 + sub * 4, gsrc + (size_t)o * 32 + sub * 4);
                    }
                }
                if (lane < V) b_cp4(dst + St::FL + lane, flags + C.flags + (size_t)tl.pk * 5 * V + lane);
            }
        }
        b_commit();
        base_out = base;
        deg_out = deg;
        return mine;
    };

    int offr[kBStages];
#pragma unroll
    for (int s = 0; s < kBStages - 1; ++s) {
        offr[s] = issue(item + s * GW, s);
        gbase[s] = base_out;
        gdeg[s] = deg_out;
    }
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kBStages - 1] = issue(item + (kBStages - 1) * GW, (slot + kBStages - 1) % kBStages);
        gbase[kBStages - 1] = base_out;
        gdeg[kBStages - 1] = deg_out;
        b_wait<kBStages - 1>();
        __syncwarp();
        const int myoff = offr[0];
        const long long base = gbase[0];
        const int deg = gdeg[0];  // warp-uniform
#pragma unroll
        for (int s = 0; s < kBStages - 1; ++s) offr[s] = offr[s + 1], gbase[s] = gbase[s + 1], gdeg[s] = gdeg[s + 1];
        if (base >= 0) {
            const uint32_t *S = ring + slot * St::WORDS;
            uint32_t *gmsg = msg + base + lane;
            bool lane_on = false;
#pragma unroll
            for (int v = 0; v < V; ++v) lane_on |= ((~S[St::FL + v]) >> lane) & 1u;
            if constexpr (!MS) {
                float ph[kBDC][V];
                uint32_t neg[V];
#pragma unroll
                for (int v = 0; v < V; ++v) neg[v] = 0u;
#pragma unroll
                for (int l = 0; l < kBDC; ++l) {
#pragma unroll
                    for (int v = 0; v < V; ++v) ph[l][v] = 0.0f;
                    if (l < deg && __shfl_sync(0xffffffffu, myoff, l) >= 0) {
                        float x[V];
                        if (FIRST) {
                            const float *mf = reinterpret_cast<const float *>(S + l * St::SEGW) + lane * V;
#pragma unroll
                            for (int v = 0; v < V; ++v) x[v] = mf[v];
                        } else {
                            Lane<V>::unpack(S[l * 32 + lane], x);
                        }
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            ph[l][v] = (XF && !FIRST) ? fabsf(x[v]) * XfScale<V>::load : phi_f(fabsf(x[v]));
                            // the sign bit: a transformed FP16 message of a strongly negative beta
                            // may round to -0
                            neg[v] |= (__float_as_uint(x[v]) >> 31) << l;
                        }
                    }
                }
                float pre[kBDC][V];
                {
                    float acc[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = 0.0f;
#pragma unroll
                    for (int l = 0; l < kBDC; ++l)
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            pre[l][v] = acc[v];
                            acc[v] += ph[l][v];
                        }
                }
                uint32_t par_all[V];
                float suf[V];
#pragma unroll
                for (int v = 0; v < V; ++v) par_all[v] = __popc(neg[v]) & 1u, suf[v] = 0.0f;
                // phi on packed pairs: two edges (V = 1) or the two frames of a lane word (V = 2)
                static_assert(V <= 2 && kBDC % 2 == 0, "pairs of edges or frames");
#pragma unroll
                for (int l = kBDC - 1; l >= 0; l -= (V == 1 ? 2 : 1)) {
                    float arg[2][V], mag[2][V];
#pragma unroll
                    for (int h = 0; h < (V == 1 ? 2 : 1); ++h)
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            arg[h][v] = pre[l - h][v] + suf[v];
                            suf[v] += ph[l - h][v];
                        }
                    if constexpr (V == 1) phi2(arg[0][0], arg[1][0], mag[0][0], mag[1][0]);
                    else phi2(arg[0][0], arg[0][1], mag[0][0], mag[0][1]);
#pragma unroll
                    for (int h = 0; h < (V == 1 ? 2 : 1); ++h) {
                        const int le = l - h;
                        const int o = __shfl_sync(0xffffffffu, myoff, le);
                        if (o >= 0) {
                            float out[V];
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const float m = fminf(mag[h][v], clip);
                                out[v] = (par_all[v] ^ ((neg[v] >> le) & 1u)) ? -m : m;
                            }
                            if (lane_on) gmsg[(size_t)o * 32] = Lane<V>::pack(out);
                        }
                    }
                }
            } else {
                uint32_t ab[kBDC], sg[kBDC];
                uint32_t min1 = 0x7f7f7f7fu, min2 = 0x7f7f7f7fu, sgn = 0u;
#pragma unroll
                for (int l = 0; l < kBDC; ++l) {
                    ab[l] = 0u;
                    sg[l] = 0u;
                    if (l < deg && __shfl_sync(0xffffffffu, myoff, l) >= 0) {
                        const uint32_t x = S[l * St::SEGW + lane];
                        const uint32_t av = __vabsss4(x);
                        sg[l] = x & 0x80808080u;
                        ab[l] = av;
                        sgn ^= sg[l];
                        min2 = __vminu4(min2, __vmaxu4(min1, av));
                        min1 = __vminu4(min1, av);
                    }
                }
#pragma unroll
                for (int l = 0; l < kBDC; ++l) {
                    if (l >= deg) break;  // warp-uniform
                    const int o = __shfl_sync(0xffffffffu, myoff, l);
                    if (o < 0) continue;  // warp-uniform
                    const uint32_t eq = __vcmpeq4(ab[l], min1);
                    const uint32_t mag = (min2 & eq) | (min1 & ~eq);
                    const uint32_t sneg = ((sgn ^ sg[l]) >> 7) & 0x01010101u;
                    if (lane_on) gmsg[(size_t)o * 32] = __vadd4(mag ^ (sneg * 0xffu), sneg);
                }
            }
        }
        __syncwarp();
        slot = (slot + 1) % kBStages;
    }
    b_wait<0>();
}

// ---------------------------------------------------------------------------
// syndrome of the decisions after the previous iteration (eq. (hrddcs)) for every
// row of the listed check-pass tiles, ORed into the package's unsat words (par):
// one thread per row, reading the packed decision words of the row's variables
// (L2-resident); a warp whose rows all belong to one tile ORs its lanes' words
// before a single atomic.  Frames already stopped are masked out.
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(256)
bsyn_kernel(const BCode *__restrict__ codes, const int *__restrict__ shtab, const uint32_t *__restrict__ hw,
            uint32_t *__restrict__ flags, const int *__restrict__ tcount, const BTile *__restrict__ tiles, int TR,
            int par) {
    const int sTR = __ffs(TR) - 1;  // TR is a power of two
    const int total = *tcount * TR;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
        const int it = base + threadIdx.x;
        int tile = -1;
        uint32_t syn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) syn[v] = 0u;
        BTile tl{0, 0, 0, 0};
        long long fl = 0;
        if (it < total) {
            tile = it >> sTR;
            tl = tiles[tile];
            const int ri = it & (TR - 1);
            const BCode C = codes[tl.code];
            fl = C.flags + (long long)tl.pk * 5 * V;
            if (ri < tl.count) {
                const int m = tl.start + ri;
                const int j = (int)fdiv((uint32_t)m, C.dp), r = m - j * C.p;
                const uint32_t *h = hw + C.hw + (size_t)tl.pk * C.N * V;
                for (int l = 0; l < C.L; ++l) {
                    const int sh = __ldg(shtab + C.tab + j * C.L + l);
                    if (sh < 0) continue;
                    int k = r + sh;
                    if (k >= C.p) k -= C.p;
#pragma unroll
                    for (int v = 0; v < V; ++v) syn[v] ^= __ldg(h + ((size_t)l * C.p + k) * V + v);
                }
#pragma unroll
                for (int v = 0; v < V; ++v) syn[v] &= ~flags[fl + v];  // running frames only
            }
        }
        const bool one_tile = __all_sync(0xffffffffu, tile == __shfl_sync(0xffffffffu, tile, 0));
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (one_tile) {
                const uint32_t any = __reduce_or_sync(0xffffffffu, syn[v]);
                if (lane == 0 && any && tile >= 0) atomicOr(flags + fl + (1 + par) * V + v, any);
            } else if (syn[v]) {
                atomicOr(flags + fl + (1 + par) * V + v, syn[v]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// variable pass over all codes
// ---------------------------------------------------------------------------
template <int V, bool MS>
struct BVnStage {
    static constexpr int MUW = MS ? 32 : 32 * V;
    static constexpr int MU = 0;
    static constexpr int AL = kBNV * MUW;
    static constexpr int HW = AL + kBNV * kBJ * 32;
    static constexpr int FL = HW + kBNV * V;
    // what the compute phase needs of the item's tile and code, written by lane 0 when the item
    // is staged: variable group g (-1: empty item), N, then the message, decision-word, flag and
    // iteration-count bases of the item's package (8-byte aligned)
    static constexpr int META = (FL + 2 * V + 1) & ~1;
    static constexpr int WORDS = (META + 2 + 8 + 3) & ~3;
};

template <int V, bool STOP, bool XF, bool MS>
__global__ void __launch_bounds__(kWarps * 32)
bvn_kernel(const BCode *__restrict__ codes, const int *__restrict__ shtab, const int *__restrict__ eotab,
           uint32_t *__restrict__ msg, const uint32_t *__restrict__ mu, uint32_t *__restrict__ hw,
           uint32_t *__restrict__ flags, int32_t *__restrict__ iters, const int *__restrict__ tcount,
           const BTile *__restrict__ tiles, int TG, float clip, int it, int par) {
    using St = BVnStage<V, MS>;
    constexpr int W = 32 * V;
    const int sTG = __ffs(TG) - 1;  // TG is a power of two
    constexpr int MU_SEGS = St::MUW / 32;
    constexpr int NSEG = kBNV * (MU_SEGS + kBJ);
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ring = smem + warp * kBStages * St::WORDS;
    const int total = *tcount * TG;
    const int GW = gridDim.x * kWarps;
    int item = blockIdx.x * kWarps + warp;

    // starts the copies of item itm; returns this lane's edge offset (lane t < kBNV * kBJ:
    // edge (variable t / kBJ, block row t % kBJ) of the item, -1 if absent)
    // the tile of the next item this warp stages, loaded one item ahead
    BTile tl_next = item < total ? b_tile(tiles, item >> sTG) : BTile{0, 0, 0, 0};
    auto issue = [&](int itm, int slot) -> int {
        int mine = -1;
        uint32_t *dst = ring + slot * St::WORDS;
        int g_meta = -1;
        const BTile tl = tl_next;
        if (itm + GW < total) tl_next = b_tile(tiles, (itm + GW) >> sTG);
        if (itm < total) {
            const int gi = itm & (TG - 1);
            if (gi < tl.count) {
                const BCode C = codes[tl.code];
                g_meta = tl.start + gi;
                if (lane == 0) {
                    dst[St::META + 1] = (uint32_t)C.N;
                    long long *mb = reinterpret_cast<long long *>(dst + St::META + 2);
                    mb[0] = C.msg + (long long)tl.pk * C.E * 32;
                    mb[1] = C.hw + (long long)tl.pk * C.N * V;
                    mb[2] = C.flags + (long long)tl.pk * 5 * V;
                    mb[3] = C.iters + (long long)tl.pk * W;
                }
                const int n0 = (tl.start + gi) * kBNV;
                const int l0 = (int)fdiv((uint32_t)n0, C.dp), k0 = n0 - l0 * C.p;
                const uint32_t *gmsg = msg + C.msg + (size_t)tl.pk * C.E * 32;
                const uint32_t *gmu = mu + C.mu + (size_t)tl.pk * C.N * St::MUW;
                const int grp = lane >> 3, sub = lane & 7;
                // lane t < kBNV * kBJ looks up edge t's offset once; the copies take it by shuffle
                if (lane < kBNV * kBJ) {
                    const int i = lane / kBJ, jj = lane - i * kBJ;
                    int l = l0, k = k0 + i;
                    if (k >= C.p) k -= C.p, ++l;
                    if (n0 + i < C.N && jj < C.J && __ldg(shtab + C.tab + jj * C.L + l) >= 0)
                        mine = __ldg(eotab + C.tab + jj * C.L + l) + k;
                }
#pragma unroll
                for (int s0 = 0; s0 < NSEG; s0 += 4) {
                    const int s = s0 + grp;
                    // the segment index is warp-uniform per group of 8 lanes; the shuffle runs on all lanes
                    const int t = s - kBNV * MU_SEGS;
                    const int o = __shfl_sync(0xffffffffu, mine, t >= 0 && t < kBNV * kBJ ? t : 0);
                    if (s < kBNV * MU_SEGS) {
                        const int i = s / MU_SEGS, h = s - i * MU_SEGS;
                        const int n = n0 + i;
                        if (n < C.N)
                            b_cp16(dst + St::MU + i * St::MUW + h * 32 + sub * 4,
                                   gmu + (size_t)n * St::MUW + h * 32 + sub * 4);
                    } else if (s < NSEG && o >= 0) {
                        b_cp16(dst + St::AL + t * 32 + sub * 4, gmsg + (size_t)o * 32 + sub * 4);
                    }
                }
                if (lane < kBNV * V) {
                    const int i = lane / V, v = lane - i * V;
                    const int n = n0 + i;
                    if (n < C.N) b_cp4(dst + St::HW + lane, hw + C.hw + ((size_t)tl.pk * C.N + n) * V + v);
                } else if (lane >= 32 - 2 * V) {
                    const int q = lane - (32 - 2 * V);
                    const int off = q < V ? q : (1 + par) * V + (q - V);
                    b_cp4(dst + St::FL + q, flags + C.flags + (size_t)tl.pk * 5 * V + off);
                }
            }
        }
        if (lane == 0) dst[St::META] = (uint32_t)g_meta;
        b_commit();
        return mine;
    };

    int offr[kBStages];
#pragma unroll
    for (int s = 0; s < kBStages - 1; ++s) offr[s] = issue(item + s * GW, s);
    int slot = 0;
    for (; item < total; item += GW) {
        offr[kBStages - 1] = issue(item + (kBStages - 1) * GW, (slot + kBStages - 1) % kBStages);
        b_wait<kBStages - 1>();
        __syncwarp();
        const int myoff = offr[0];
#pragma unroll
        for (int s = 0; s < kBStages - 1; ++s) offr[s] = offr[s + 1];
        const uint32_t *S = ring + slot * St::WORDS;
        const int g = (int)S[St::META];  // warp-uniform
        if (g >= 0) {
            const int CN = (int)S[St::META + 1];
            const long long *mb = reinterpret_cast<const long long *>(S + St::META + 2);
            const long long msg_b = mb[0], hw_b = mb[1], fl_b = mb[2], it_b = mb[3];
            uint32_t *gmsg = msg + msg_b + lane;
            uint32_t frozen[V];
            bool lane_on = false;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                uint32_t dn = S[St::FL + v];
                if (STOP) {
                    const uint32_t newly = ~dn & ~S[St::FL + V + v];
                    if (g == 0 && lane == 0) {
                        uint32_t *F = flags + fl_b;
                        if (newly) {
                            F[v] = dn | newly;
                            for (uint32_t b = newly; b; b &= b - 1) {
                                const int ln = __ffs(b) - 1;
                                iters[it_b + ln * V + v] = it - 1;
                            }
                        }
                        F[(1 + (par ^ 1)) * V + v] = 0u;
                    }
                    dn |= newly;
                }
                frozen[v] = dn;
                lane_on |= ((~dn) >> lane) & 1u;
            }
            const int n0 = g * kBNV;
#pragma unroll
            for (int i = 0; i < kBNV; ++i) {
                const int n = n0 + i;
                if (n >= CN) break;
                int eo[kBJ];  // the item's edge offsets, -1 absent (warp-uniform)
#pragma unroll
                for (int jj = 0; jj < kBJ; ++jj) eo[jj] = __shfl_sync(0xffffffffu, myoff, i * kBJ + jj);
                uint32_t outb[V];
                if constexpr (!MS) {
                    float m[V], aj[kBJ][V], tot[V];
                    const float *mf = reinterpret_cast<const float *>(S + St::MU + i * St::MUW) + lane * V;
#pragma unroll
                    for (int v = 0; v < V; ++v) m[v] = mf[v], tot[v] = mf[v];
#pragma unroll
                    for (int jj = 0; jj < kBJ; ++jj) {
#pragma unroll
                        for (int v = 0; v < V; ++v) aj[jj][v] = 0.0f;
                        if (eo[jj] >= 0) {
                            Lane<V>::unpack(S[St::AL + (i * kBJ + jj) * 32 + lane], aj[jj]);
#pragma unroll
                            for (int v = 0; v < V; ++v) tot[v] += aj[jj][v];
                        }
                    }
                    float bj[kBJ][V];
#pragma unroll
                    for (int jj = 0; jj < kBJ; ++jj)
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            float s = m[v];
#pragma unroll
                            for (int j2 = 0; j2 < kBJ; ++j2)
                                if (j2 != jj) s += aj[j2][v];
                            bj[jj][v] = clipf(s, clip);
                        }
                    if constexpr (XF) {
                        // phi of |beta| on packed pairs (two edges, or the two frames of a lane word)
                        float f[kBJ][V];
                        if constexpr (V == 2) {
#pragma unroll
                            for (int jj = 0; jj < kBJ; ++jj)
                                phi_fin2(fabsf(bj[jj][0]), fabsf(bj[jj][1]), f[jj][0], f[jj][1]);
                        } else {
                            static_assert(kBJ % 2 == 0, "edge pairs");
#pragma unroll
                            for (int jj = 0; jj < kBJ; jj += 2)
                                phi_fin2(fabsf(bj[jj][0]), fabsf(bj[jj + 1][0]), f[jj][0], f[jj + 1][0]);
                        }
#pragma unroll
                        for (int jj = 0; jj < kBJ; ++jj)
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const float t = f[jj][v] * XfScale<V>::store;
                                bj[jj][v] = bj[jj][v] < 0.0f ? -t : t;
                            }
                    }
#pragma unroll
                    for (int jj = 0; jj < kBJ; ++jj) {
                        if (eo[jj] < 0) continue;
                        if (lane_on) gmsg[(size_t)eo[jj] * 32] = Lane<V>::pack(bj[jj]);
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) outb[v] = __ballot_sync(0xffffffffu, clipf(tot[v], clip) < 0.0f);
                } else {
                    const uint32_t qw = S[St::MU + i * St::MUW + lane];
                    uint32_t aw[kBJ];
                    int tot[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) tot[v] = sbyte(qw, v);
#pragma unroll
                    for (int jj = 0; jj < kBJ; ++jj) {
                        aw[jj] = 0u;
                        if (eo[jj] >= 0) {
                            aw[jj] = S[St::AL + (i * kBJ + jj) * 32 + lane];
#pragma unroll
                            for (int v = 0; v < 4; ++v) tot[v] += sbyte(aw[jj], v);
                        }
                    }
                    if (lane_on) {
#pragma unroll
                        for (int jj = 0; jj < kBJ; ++jj) {
                            if (eo[jj] < 0) continue;
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
#pragma unroll
                    for (int v = 0; v < V; ++v) outb[v] = __ballot_sync(0xffffffffu, tot[v] < 0);
                }
                if (lane == 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const uint32_t old = S[St::HW + i * V + v];
                        hw[hw_b + (size_t)n * V + v] = (outb[v] & ~frozen[v]) | (old & frozen[v]);
                    }
                }
            }
        }
        __syncwarp();
        slot = (slot + 1) % kBStages;
    }
    b_wait<0>();
}

// ---------------------------------------------------------------------------
// Frame-level compaction.  Early stop frees lanes, but a package of W frames is
// visited until its slowest frame stops.  After iteration K every code whose
// running frames are few enough moves them, densely and in frame order, into its
// second package area (entered in the code table as code nc + c): messages,
// channel LLRs, decision bits; the first area's frames are then all marked done,
// and the tile lists pick up the second area.  map[k] is the frame (slot of the
// first area) now in slot k of the second; its outputs are scattered back at the
// end.  Codes whose running frames exceed limit of their frames are left as they are.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int b_block_sum(int x, int *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += sh[w];
    return t;
}

// one block per code: count, decide, number the running frames in frame order, retire the first area
__global__ void __launch_bounds__(1024)
bcompact_plan_kernel(const BCode *__restrict__ codes, uint32_t *__restrict__ flags, int *__restrict__ map,
                     int *__restrict__ moved, int V, float limit) {
    __shared__ int sh[32];
    __shared__ int s_base;
    const int c = blockIdx.x;
    const BCode C = codes[c];
    const int W = 32 * V, frames = C.P * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *F = flags + C.flags;
    auto running = [&](int f) -> bool {
        const int pk = f / W, ln = (f % W) / V, v = f % V;
        const uint32_t *b = F + (size_t)pk * 5 * V;
        return !((b[v] >> ln) & 1u) && ((b[3 * V + v] >> ln) & 1u);
    };
    int cnt = 0, val = 0;
    for (int f = threadIdx.x; f < frames; f += blockDim.x) {
        const int pk = f / W, ln = (f % W) / V, v = f % V;
        val += (F[(size_t)pk * 5 * V + 3 * V + v] >> ln) & 1u;
        cnt += running(f) ? 1 : 0;
    }
    const int R = b_block_sum(cnt, sh);
    const int valid = b_block_sum(val, sh);
    if (R == 0 || (float)R > limit * (float)valid) {
        if (threadIdx.x == 0) moved[c] = 0;
        return;
    }
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int f0 = 0; f0 < frames; f0 += blockDim.x) {
        const int f = f0 + threadIdx.x;
        const bool r = f < frames && running(f);
        const uint32_t bal = __ballot_sync(0xffffffffu, r);
        __syncthreads();
        if (lane == 0) sh[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += sh[w];
            all += sh[w];
        }
        if (r) map[C.map + s_base + before + __popc(bal & ((1u << lane) - 1u))] = f;
        __syncthreads();
        if (threadIdx.x == 0) s_base += all;
        __syncthreads();
    }
    // every frame of the first area is now done (stopped, or moved on)
    for (int i = threadIdx.x; i < C.P * V; i += blockDim.x) F[(size_t)(i / V) * 5 * V + i % V] = 0xffffffffu;
    if (threadIdx.x == 0) moved[c] = R;
}

// the second area of code c: messages (one thread per destination lane word), channel LLRs
// (per destination element) and decision words (one warp per destination word, a ballot of
// the moved frames' bits), flags (done past the moved frames, unsat and fin cleared)
template <int V, bool MS>
__global__ void __launch_bounds__(256)
bcompact_gather_kernel(const BCode *__restrict__ codes, uint32_t *__restrict__ msg, uint32_t *__restrict__ mu,
                       uint32_t *__restrict__ hw, uint32_t *__restrict__ flags, const int *__restrict__ map,
                       const int *__restrict__ moved, int nc) {
    constexpr int W = 32 * V;
    constexpr int EB = 32 / V;  // bits of one message element
    const int c = blockIdx.y;
    const int R = moved[c];
    if (R == 0) return;
    const BCode A = codes[c], B = codes[nc + c];
    const int P2 = (R + W - 1) / W;
    const int *mp = map + A.map;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // messages: word (pk2, e, lane2)
    const long long nmsg = (long long)P2 * A.E * 32;
    for (long long i = tid; i < nmsg; i += stride) {
        const int lane2 = (int)(i & 31);
        const long long pe = i >> 5;
        const int e = (int)(pe % A.E), pk2 = (int)(pe / A.E);
        uint32_t w = 0u;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int k = pk2 * W + lane2 * V + v;
            if (k >= R) break;
            const int f = mp[k];
            const int pk = f / W, ln = (f % W) / V, vs = f % V;
            const uint32_t src = msg[A.msg + ((size_t)pk * A.E + e) * 32 + ln];
            const uint32_t sub = V == 1 ? src : (src >> (vs * EB)) & ((1u << EB) - 1u);
            w |= sub << (v * EB);
        }
        msg[B.msg + ((size_t)pk2 * A.E + e) * 32 + lane2] = w;
    }
    // channel LLRs: element (pk2, n, j) of [P][N][W] (floats; int8 for min-sum)
    const long long nmu = (long long)P2 * A.N * W;
    for (long long i = tid; i < nmu; i += stride) {
        const int j = (int)(i % W);
        const long long pn = i / W;
        const int n = (int)(pn % A.N), pk2 = (int)(pn / A.N);
        const int k = pk2 * W + j;
        if (k >= R) continue;
        const int f = mp[k];
        const size_t si = ((size_t)(f / W) * A.N + n) * W + (f % W), di = ((size_t)pk2 * A.N + n) * W + j;
        if (MS) reinterpret_cast<int8_t *>(mu + B.mu)[di] = reinterpret_cast<const int8_t *>(mu + A.mu)[si];
        else reinterpret_cast<float *>(mu + B.mu)[di] = reinterpret_cast<const float *>(mu + A.mu)[si];
    }
    // decision words: one warp per destination word (pk2, n, v)
    const long long nhw = (long long)P2 * A.N * V;
    const int lane = threadIdx.x & 31;
    for (long long wi = tid >> 5; wi < nhw; wi += stride >> 5) {
        const int v = (int)(wi % V);
        const long long pn = wi / V;
        const int n = (int)(pn % A.N), pk2 = (int)(pn / A.N);
        const int k = pk2 * W + lane * V + v;
        uint32_t bit = 0u;
        if (k < R) {
            const int f = mp[k];
            bit = (hw[A.hw + ((size_t)(f / W) * A.N + n) * V + f % V] >> ((f % W) / V)) & 1u;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bit != 0u);
        if (lane == 0) hw[B.hw + ((size_t)pk2 * A.N + n) * V + v] = word;
    }
    // flags of the second area
    for (long long i = tid; i < (long long)A.P * V; i += stride) {
        const int pk2 = (int)(i / V), v = (int)(i % V);
        uint32_t valid = 0u;
        for (int ln = 0; ln < 32; ++ln)
            if (pk2 * W + ln * V + v < R) valid |= 1u << ln;
        uint32_t *b = flags + B.flags + (size_t)pk2 * 5 * V;
        b[v] = ~valid;
        b[V + v] = 0u;
        b[2 * V + v] = 0u;
        b[3 * V + v] = valid;
        b[4 * V + v] = 0u;
    }
}

// every package of the second areas holds no frame (done), before a decode
__global__ void bsecond_init_kernel(const BCode *__restrict__ codes, uint32_t *__restrict__ flags, int *__restrict__ moved,
                                    int nc, int V) {
    const int c = blockIdx.x;
    const BCode B = codes[nc + c];
    for (int i = threadIdx.x; i < B.P * 5 * V; i += blockDim.x) flags[B.flags + i] = (i % (5 * V)) < V ? 0xffffffffu : 0u;
    if (threadIdx.x == 0) moved[c] = 0;
}

// the syndrome of the moved frames' last decisions (eq. (hrddcs)) into the fin words of the second
// areas: one thread per (package, row) of the packages holding moved frames
__global__ void __launch_bounds__(256)
bsec_syndrome_kernel(const BCode *__restrict__ codes, const int *__restrict__ shtab, const uint32_t *__restrict__ hw,
                     uint32_t *__restrict__ flags, const int *__restrict__ moved, int nc, int V) {
    const int c = blockIdx.y;
    const int R = moved[c];
    if (R == 0) return;
    const BCode B = codes[nc + c];
    const int W = 32 * V;
    const long long total = (long long)((R + W - 1) / W) * B.M;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int pk2 = (int)(i / B.M), m = (int)(i % B.M);
        const int j = (int)fdiv((uint32_t)m, B.dp), r = m - j * B.p;
        const uint32_t *h = hw + B.hw + (size_t)pk2 * B.N * V;
        uint32_t syn[4] = {0u, 0u, 0u, 0u};
        for (int l = 0; l < B.L; ++l) {
            const int sh = __ldg(shtab + B.tab + j * B.L + l);
            if (sh < 0) continue;
            int k = r + sh;
            if (k >= B.p) k -= B.p;
            for (int v = 0; v < V; ++v) syn[v] ^= __ldg(h + ((size_t)l * B.p + k) * V + v);
        }
        for (int v = 0; v < V; ++v)
            if (syn[v]) atomicOr(flags + B.flags + (size_t)pk2 * 5 * V + 4 * V + v, syn[v]);
    }
}

// the moved frames' decisions, iteration counts (as the frames stopped, else max_iter) and ok flags
// (last decisions satisfy every check) go to their rows of the caller's outputs (pointer arrays per
// code, entries may be NULL)
__global__ void __launch_bounds__(256)
bscatter_kernel(const BCode *__restrict__ codes, const uint32_t *__restrict__ hw, const uint32_t *__restrict__ flags,
                const int32_t *__restrict__ iters, const int *__restrict__ map, const int *__restrict__ moved, int nc,
                int V, int max_iter, uint8_t *const *__restrict__ hard, int32_t *const *__restrict__ itout,
                int32_t *const *__restrict__ okout) {
    const int c = blockIdx.y;
    const int R = moved[c];
    if (R == 0) return;
    const BCode A = codes[c], B = codes[nc + c];
    const int W = 32 * V;
    const int *mp = map + A.map;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = tid; i < R; i += stride) {
        const int f = mp[i];
        const int pk2 = (int)i / W, ln = ((int)i % W) / V, v = (int)i % V;
        const uint32_t *fl = flags + B.flags + (size_t)pk2 * 5 * V;
        const bool stopped = (fl[v] >> ln) & 1u;
        if (itout && itout[c]) itout[c][f] = stopped ? iters[B.iters + i] : max_iter;
        if (okout && okout[c]) okout[c][f] = ((fl[4 * V + v] >> ln) & 1u) ? 0 : 1;
    }
    if (!hard || !hard[c]) return;
    uint8_t *h = hard[c];
    const long long total = (long long)R * A.N;
    for (long long i = tid; i < total; i += stride) {
        const int k = (int)(i / A.N), n = (int)(i % A.N);
        const uint32_t w = hw[B.hw + ((size_t)(k / W) * A.N + n) * V + k % V];
        h[(size_t)mp[k] * A.N + n] = (uint8_t)((w >> ((k % W) / V)) & 1u);
    }
}

// ---------------------------------------------------------------------------
// tile lists of the packages with a running frame, over all codes
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
btiles_kernel(const BCode *__restrict__ codes, const int *__restrict__ pair_code, const int *__restrict__ pair_pk,
              int npairs, const uint32_t *__restrict__ flags, int V, int TR, int TG, int *__restrict__ cn_count,
              BTile *__restrict__ cn_tiles, int *__restrict__ vn_count, BTile *__restrict__ vn_tiles, int first) {
    __shared__ int ws_c[32], ws_v[32];
    __shared__ int base_c, base_v;
    if (threadIdx.x == 0) base_c = base_v = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p0 = 0; p0 < npairs; p0 += blockDim.x) {
        const int q = p0 + threadIdx.x;
        int nc = 0, nv = 0, code = 0, pk = 0;
        if (q < npairs) {
            code = pair_code[q];
            pk = pair_pk[q];
            const BCode C = codes[code];
            bool on = first != 0;
            for (int v = 0; v < V && !on; ++v) on = ~flags[C.flags + (size_t)pk * 5 * V + v] != 0u;
            if (on) {
                nc = (C.M + TR - 1) / TR;
                nv = ((C.N + kBNV - 1) / kBNV + TG - 1) / TG;
            }
        }
        // inclusive warp scans of the tile counts
        int sc = nc, sv = nv;
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, sc, o), b = __shfl_up_sync(0xffffffffu, sv, o);
            if (lane >= o) sc += a, sv += b;
        }
        if (lane == 31) ws_c[warp] = sc, ws_v[warp] = sv;
        __syncthreads();
        int pc = 0, pv = 0, tc = 0, tv = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) pc += ws_c[w], pv += ws_v[w];
            tc += ws_c[w];
            tv += ws_v[w];
        }
        const int oc = base_c + pc + sc - nc, ov = base_v + pv + sv - nv;
        if (q < npairs) {
            const BCode C = codes[code];
            for (int t = 0; t < nc; ++t) {
                const int start = t * TR;
                cn_tiles[oc + t] = BTile{code, pk, start, min(TR, C.M - start)};
            }
            const int G = (C.N + kBNV - 1) / kBNV;
            for (int t = 0; t < nv; ++t) {
                const int start = t * TG;
                vn_tiles[ov + t] = BTile{code, pk, start, min(TG, G - start)};
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_c += tc, base_v += tv;
        __syncthreads();
    }
    if (threadIdx.x == 0) *cn_count = base_c, *vn_count = base_v;
}

}  // namespace ldpc

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using namespace ldpc;

struct ldpc_batch_s {
    int ncodes = 0, V = 1;
    ldpc_decode_opts o;
    std::unique_ptr<ldpc_code_s[]> views;  // per-code views into the shared workspace
    int nviews = 0;
    std::vector<BCode> hcodes;
    BCode *codes = nullptr;
    int *shtab = nullptr, *eotab = nullptr;
    int *pair_code = nullptr, *pair_pk = nullptr;
    int npairs = 0;
    int *counts = nullptr;  // [2]: cn, vn tile counts
    BTile *cn_tiles = nullptr, *vn_tiles = nullptr;
    size_t max_cn_tiles = 0, max_vn_tiles = 0;
    void *msg = nullptr, *mu = nullptr;
    uint32_t *hw = nullptr, *flags = nullptr;
    int32_t *iters = nullptr;  // per code: [cap] iterations, then [cap] ok flags
    float *post = nullptr;
    int *act = nullptr;
    size_t hw_words = 0, flags_words = 0, iters_total = 0;
    int TR = 0, TG = 0;
    bool tuned = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double tune_ms[3] = {0, 0, 0};
    // frame-level compaction: entries ncodes .. 2 ncodes - 1 of the code table are the codes'
    // second package areas; after iteration K a code's running frames move there when they are
    // at most `limit` of its frames
    int *map = nullptr;     // per code: second-area slot -> frame
    int *moved = nullptr;   // [ncodes] frames moved by the last decode
    uint8_t **d_hard = nullptr;   // device copies of the caller's output pointer arrays
    int32_t **d_iters = nullptr, **d_ok = nullptr;
    void **h_ptrs = nullptr;      // pinned staging of those arrays [3][ncodes]
    cudaEvent_t ptr_ev = nullptr; // recorded after their copy; waited on before the next overwrite
    int K = -1;             // compaction after iteration K (0: never, -1: chosen by the autotuner)
    float limit = 0.75f;
    double tune_k_ms[4] = {0, 0, 0, 0};  // full-decode times of the compaction candidates
    int sms = 1;
};

namespace ldpc {

template <typename K>
static int b_blocks(K kernel, size_t smem) {
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, kWarps * 32, smem);
    return (bps < 1 ? 1 : bps) * (sms < 1 ? 1 : sms);
}

template <int V, bool XF, bool MS>
static void b_cn(ldpc_batch b, bool first, bool syn, int par, cudaStream_t s) {
    if (syn) {
        // the syndrome of the decisions after it - 1 iterations, before the check pass
        static int sblocks = 0;
        if (!sblocks) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            sblocks = (sms > 0 ? sms : 1) * 8;
        }
        bsyn_kernel<V><<<sblocks, 256, 0, s>>>(b->codes, b->shtab, b->hw, b->flags, b->counts, b->cn_tiles, b->TR,
                                               par);
    }
#define B_CN(FIRSTV)                                                                                               \
    do {                                                                                                           \
        auto k = bcn_kernel<V, XF, MS, FIRSTV>;                                                                    \
        const size_t sm = (size_t)kWarps * kBStages * BCnStage<V, FIRSTV, MS>::WORDS * 4;                          \
        static int blocks = 0;                                                                                     \
        if (!blocks) blocks = b_blocks(k, sm);                                                                     \
        k<<<blocks, kWarps * 32, sm, s>>>(b->codes, b->shtab, b->eotab, (uint32_t *)b->msg, (const uint32_t *)b->mu, \
                                          b->flags, b->counts, b->cn_tiles, b->TR, b->o.clip);                     \
    } while (0)
    if (first) B_CN(true);
    else B_CN(false);
#undef B_CN
}

template <int V, bool XF, bool MS>
static void b_vn(ldpc_batch b, bool stop, int it, int par, cudaStream_t s) {
#define B_VN(STOPV)                                                                                                  \
    do {                                                                                                             \
        auto k = bvn_kernel<V, STOPV, XF, MS>;                                                                       \
        const size_t sm = (size_t)kWarps * kBStages * BVnStage<V, MS>::WORDS * 4;                                    \
        static int blocks = 0;                                                                                       \
        if (!blocks) blocks = b_blocks(k, sm);                                                                       \
        k<<<blocks, kWarps * 32, sm, s>>>(b->codes, b->shtab, b->eotab, (uint32_t *)b->msg, (const uint32_t *)b->mu, \
                                          b->hw, b->flags, b->iters, b->counts + 1, b->vn_tiles, b->TG, b->o.clip,  \
                                          it, par);                                                                  \
    } while (0)
    if (stop) B_VN(true);
    else B_VN(false);
#undef B_VN
}

static void b_tiles(ldpc_batch b, bool first, cudaStream_t s) {
    btiles_kernel<<<1, 1024, 0, s>>>(b->codes, b->pair_code, b->pair_pk, b->npairs, b->flags, b->V, b->TR, b->TG,
                                     b->counts, b->cn_tiles, b->counts + 1, b->vn_tiles, first ? 1 : 0);
}

// one iteration of the shared loop
static void b_iteration(ldpc_batch b, int it, cudaStream_t s) {
    const bool first = it == 1, syn = b->o.early_stop && it >= 2;
    const int par = it & 1;
    if (b->o.algo == LDPC_ALGO_MS) {
        b_cn<4, false, true>(b, first, syn, par, s);
        b_vn<4, false, true>(b, syn, it, par, s);
    } else if (b->o.msg == LDPC_MSG_F16) {
        b_cn<2, true, false>(b, first, syn, par, s);
        b_vn<2, true, false>(b, syn, it, par, s);
    } else {
        b_cn<1, true, false>(b, first, syn, par, s);
        b_vn<1, true, false>(b, syn, it, par, s);
    }
    if (b->o.early_stop && b->K > 0 && it == b->K && it < b->o.max_iter) {
        // frame-level compaction (the tile rebuild below lists the second areas' packages)
        bcompact_plan_kernel<<<b->ncodes, 1024, 0, s>>>(b->codes, b->flags, b->map, b->moved, b->V, b->limit);
        const dim3 grd((unsigned)(b->sms * 2), (unsigned)b->ncodes);
        if (b->o.algo == LDPC_ALGO_MS)
            bcompact_gather_kernel<4, true><<<grd, 256, 0, s>>>(b->codes, (uint32_t *)b->msg, (uint32_t *)b->mu, b->hw,
                                                               b->flags, b->map, b->moved, b->ncodes);
        else if (b->o.msg == LDPC_MSG_F16)
            bcompact_gather_kernel<2, false><<<grd, 256, 0, s>>>(b->codes, (uint32_t *)b->msg, (uint32_t *)b->mu, b->hw,
                                                                b->flags, b->map, b->moved, b->ncodes);
        else
            bcompact_gather_kernel<1, false><<<grd, 256, 0, s>>>(b->codes, (uint32_t *)b->msg, (uint32_t *)b->mu, b->hw,
                                                                b->flags, b->map, b->moved, b->ncodes);
        count_launch(2);
    }
    if (b->o.early_stop && it < b->o.max_iter) b_tiles(b, false, s);
    count_launch((b->o.early_stop && it < b->o.max_iter ? 3 : 2) + (syn ? 1 : 0));
}

static void b_loop(ldpc_batch b, int iters, cudaStream_t s) {
    for (int it = 1; it <= iters; ++it) b_iteration(b, it, s);
}

}  // namespace ldpc

// implemented in qc_decode.cu
namespace ldpc {
ldpc_status qc_init_flags(ldpc_code c, int gamma, int V, cudaStream_t s);
ldpc_status qc_finish(ldpc_code c, int gamma, const ldpc_decode_opts &o, cudaStream_t s);
}  // namespace ldpc

extern "C" {

ldpc_status ldpc_batch_create(const ldpc_code *codes, int32_t ncodes, const int32_t *gammas,
                              const ldpc_decode_opts *opts, ldpc_batch *out) {
    if (!out || !codes || !gammas || !opts || ncodes < 1 || ncodes > 4096) {
        set_error("need codes, gammas, opts, out and 1 <= ncodes <= 4096");
        return LDPC_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < ncodes; ++i)
        if (!codes[i] || codes[i]->sparse) {
            set_error("code %d: batches take QC codes", i);
            return codes[i] ? LDPC_EUNSUPPORTED : LDPC_EINVAL;
        }
    const ldpc_decode_opts &o = *opts;
    if (o.max_iter < 1 || o.max_iter > 100000 ||
        !((o.algo == LDPC_ALGO_SP && (o.msg == LDPC_MSG_F32 || o.msg == LDPC_MSG_F16)) ||
          (o.algo == LDPC_ALGO_MS && o.msg == LDPC_MSG_I8)) ||
        !(o.clip > 0.0f) || o.clip > 60000.0f) {
        set_error("batches take sum-product (F32/F16) or integer min-sum (I8), 1 <= max_iter, 0 < clip <= 60000");
        return LDPC_EUNSUPPORTED;
    }
    ldpc_batch b = new (std::nothrow) ldpc_batch_s();
    if (!b) {
        set_error("host allocation failed");
        return LDPC_ENOMEM;
    }
    b->ncodes = ncodes;
    b->o = o;
    b->V = lanes_per_word(o.msg);
    const int V = b->V, W = 32 * V;
    // sizes and offsets
    size_t msg_w = 0, mu_w = 0, hw_w = 0, fl_w = 0, it_n = 0, post_n = 0;
    std::vector<int> hsh, heo, pc, pp;
    size_t max_ct = 0, max_vt = 0;
    b->hcodes.resize(2 * (size_t)ncodes);
    size_t map_n = 0;
    for (int i = 0; i < ncodes; ++i) {
        const ldpc_code c = codes[i];
        if (!c || gammas[i] < 1) {
            delete b;
            set_error("code %d is NULL or has gamma < 1", i);
            return LDPC_EINVAL;
        }
        if (c->d.J > kBJ || c->d.L > kBDC) {
            delete b;
            set_error("code %d: batches take J <= %d and L <= %d", i, kBJ, kBDC);
            return LDPC_EUNSUPPORTED;
        }
        const int P = (gammas[i] + W - 1) / W;
        BCode &bc = b->hcodes[i];
        bc.J = c->d.J; bc.L = c->d.L; bc.p = c->d.p; bc.N = c->d.N; bc.M = c->d.M; bc.E = c->d.E;
        bc.P = P; bc.gamma = gammas[i];
        bc.dp = fast_div((uint32_t)c->d.p);
        bc.tab = (int)hsh.size();
        for (int q = 0; q < c->d.J * c->d.L; ++q) hsh.push_back(c->d.shift[q]), heo.push_back(c->d.eoff[q]);
        bc.msg = (long long)msg_w;
        bc.mu = (long long)mu_w;
        bc.hw = (long long)hw_w;
        bc.flags = (long long)fl_w;
        bc.iters = (long long)it_n;
        msg_w += (size_t)P * c->d.E * 32;
        mu_w += (size_t)P * c->d.N * (o.algo == LDPC_ALGO_MS ? 32 : W);
        hw_w += (size_t)P * c->d.N * V;
        fl_w += (size_t)P * 5 * V;
        it_n += (size_t)P * W * 2;  // iterations, then ok flags (the single-code layout)
        post_n += (size_t)P * c->d.N * W;
        for (int pk = 0; pk < P; ++pk) pc.push_back(i), pp.push_back(pk);
        max_ct += (size_t)P * c->d.M;                    // tiles of one row each at most
        max_vt += (size_t)P * ((c->d.N + kBNV - 1) / kBNV);
        bc.map = (long long)map_n;
        map_n += (size_t)P * W;
    }
    // the second package areas (frame-level compaction): entries ncodes + i, same geometry
    for (int i = 0; i < ncodes; ++i) {
        const ldpc_code c = codes[i];
        BCode bc = b->hcodes[i];
        const int P = bc.P;
        bc.gamma = 0;
        bc.msg = (long long)msg_w;
        bc.mu = (long long)mu_w;
        bc.hw = (long long)hw_w;
        bc.flags = (long long)fl_w;
        bc.iters = (long long)it_n;
        msg_w += (size_t)P * c->d.E * 32;
        mu_w += (size_t)P * c->d.N * (o.algo == LDPC_ALGO_MS ? 32 : W);
        hw_w += (size_t)P * c->d.N * V;
        fl_w += (size_t)P * 5 * V;
        it_n += (size_t)P * W * 2;
        b->hcodes[ncodes + i] = bc;
        for (int pk = 0; pk < P; ++pk) pc.push_back(ncodes + i), pp.push_back(pk);
        max_ct += (size_t)P * c->d.M;
        max_vt += (size_t)P * ((c->d.N + kBNV - 1) / kBNV);
    }
    b->npairs = (int)pc.size();
    auto fail = [&](const char *what) {
        cudaGetLastError();
        ldpc_batch_destroy(b);
        set_error("device allocation failed (%s)", what);
        return LDPC_ENOMEM;
    };
    if (cudaMalloc(&b->msg, msg_w * 4)) return fail("messages");
    if (cudaMalloc(&b->mu, mu_w * 4)) return fail("channel LLRs");
    if (cudaMalloc(&b->hw, hw_w * 4)) return fail("hard words");
    if (cudaMalloc(&b->flags, fl_w * 4)) return fail("flags");
    if (cudaMalloc(&b->iters, it_n * 4)) return fail("iterations");
    if (cudaMalloc(&b->codes, sizeof(BCode) * 2 * ncodes)) return fail("code table");
    if (cudaMalloc(&b->map, (map_n ? map_n : 1) * sizeof(int)) || cudaMalloc(&b->moved, ncodes * sizeof(int)) ||
        cudaMalloc(&b->d_hard, ncodes * sizeof(void *)) || cudaMalloc(&b->d_iters, ncodes * sizeof(void *)) ||
        cudaMalloc(&b->d_ok, ncodes * sizeof(void *)))
        return fail("compaction tables");
    if (cudaHostAlloc(&b->h_ptrs, 3 * (size_t)ncodes * sizeof(void *), cudaHostAllocDefault) ||
        cudaEventCreateWithFlags(&b->ptr_ev, cudaEventDisableTiming))
        return fail("output pointer staging");
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        if (b->sms < 1) b->sms = 1;
    }
    if (cudaMalloc(&b->shtab, hsh.size() * 4) || cudaMalloc(&b->eotab, heo.size() * 4)) return fail("shift tables");
    if (cudaMalloc(&b->pair_code, pc.size() * 4) || cudaMalloc(&b->pair_pk, pp.size() * 4)) return fail("pairs");
    if (cudaMalloc(&b->counts, 2 * sizeof(int))) return fail("counts");
    if (cudaMalloc(&b->cn_tiles, max_ct * sizeof(BTile)) || cudaMalloc(&b->vn_tiles, max_vt * sizeof(BTile)))
        return fail("tiles");
    b->max_cn_tiles = max_ct;
    b->max_vn_tiles = max_vt;
    b->hw_words = hw_w;
    b->flags_words = fl_w;
    b->iters_total = it_n;
    if (cudaMemcpy(b->codes, b->hcodes.data(), sizeof(BCode) * 2 * ncodes, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->shtab, hsh.data(), hsh.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->eotab, heo.data(), heo.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->pair_code, pc.data(), pc.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(b->pair_pk, pp.data(), pp.size() * 4, cudaMemcpyHostToDevice))
        return fail("table upload");
    // per-code views: the single-code pack / finish / unpack kernels run on them
    b->views.reset(new (std::nothrow) ldpc_code_s[2 * (size_t)ncodes]);
    if (!b->views) return fail("host allocation");
    b->nviews = 2 * ncodes;
    for (int i = 0; i < 2 * ncodes; ++i) {
        ldpc_code_s &v = b->views[i];
        const BCode &bc = b->hcodes[i];
        v.d = codes[i % ncodes]->d;
        v.device = codes[i % ncodes]->device;
        v.rate = codes[i % ncodes]->rate;
        v.noms = nullptr;
        v.ws.gamma_cap = (size_t)bc.P * W;
        v.ws.msg = (uint32_t *)b->msg + bc.msg;
        v.ws.mu = (uint32_t *)b->mu + bc.mu;
        v.ws.hw = b->hw + bc.hw;
        v.ws.flags = b->flags + bc.flags;
        v.ws.iters = b->iters + bc.iters;  // ok flags follow at + gamma_cap
        v.ws.post = nullptr;
    }
    *out = b;
    return LDPC_OK;
}

ldpc_status ldpc_batch_destroy(ldpc_batch b) {
    if (!b) return LDPC_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->msg); cudaFree(b->mu); cudaFree(b->hw); cudaFree(b->flags); cudaFree(b->iters);
    cudaFree(b->codes); cudaFree(b->shtab); cudaFree(b->eotab); cudaFree(b->pair_code); cudaFree(b->pair_pk);
    cudaFree(b->counts); cudaFree(b->cn_tiles); cudaFree(b->vn_tiles);
    cudaFree(b->map); cudaFree(b->moved); cudaFree(b->d_hard); cudaFree(b->d_iters); cudaFree(b->d_ok);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    if (b->ptr_ev) cudaEventDestroy(b->ptr_ev);
    for (int i = 0; i < b->nviews; ++i) b->views[i].ws = DecodeWs();  // borrowed
    delete b;
    return LDPC_OK;
}

}  // extern "C"

namespace ldpc {

// pack every code's frames and reset its state; the initial tile list covers every package
static ldpc_status b_prepare(ldpc_batch b, const float *const *llr, cudaStream_t s) {
    for (int i = 0; i < b->ncodes; ++i) {
        ldpc_status st = qc_pack_llr(&b->views[i], llr[i], b->hcodes[i].gamma, b->o, s);
        if (st != LDPC_OK) return st;
        st = qc_init_flags(&b->views[i], b->hcodes[i].gamma, b->V, s);
        if (st != LDPC_OK) return st;
    }
    LDPC_CUDA_TRY(cudaMemsetAsync(b->hw, 0, b->hw_words * 4, s));
    bsecond_init_kernel<<<b->ncodes, 256, 0, s>>>(b->codes, b->flags, b->moved, b->ncodes, b->V);
    count_launch();
    b_tiles(b, true, s);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// autotuner: rows per check-pass tile and variable groups per variable-pass tile (powers of two:
// the passes split work items by shifts)
static ldpc_status b_tune(ldpc_batch b, const float *const *llr, cudaStream_t s) {
    const int cand[3][2] = {{16, 8}, {64, 32}, {256, 128}};
    const int iters = b->o.max_iter < 3 ? b->o.max_iter : 3;
    cudaEvent_t e0, e1;
    LDPC_CUDA_TRY(cudaEventCreate(&e0));
    LDPC_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e30;
    int bi = 1;
    for (int q = 0; q < 3; ++q) {
        b->TR = cand[q][0];
        b->TG = cand[q][1];
        ldpc_status st = b_prepare(b, llr, s);
        if (st != LDPC_OK) return st;
        b_loop(b, 1, s);  // warm-up of this configuration
        st = b_prepare(b, llr, s);
        if (st != LDPC_OK) return st;
        LDPC_CUDA_TRY(cudaEventRecord(e0, s));
        b_loop(b, iters, s);
        LDPC_CUDA_TRY(cudaEventRecord(e1, s));
        LDPC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        LDPC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        b->tune_ms[q] = ms;
        if (ms < best) best = ms, bi = q;
    }
    b->TR = cand[bi][0];
    b->TG = cand[bi][1];
    // the compaction point: whole decodes without it and with it after iterations 8, 12, 16
    if (b->K < 0) {
        const int kc[4] = {0, 8, 12, 16};
        double kbest = 1e30;
        int kb = 0;
        for (int q = 0; q < 4; ++q) {
            if (kc[q] > 0 && (!b->o.early_stop || kc[q] >= b->o.max_iter)) continue;
            b->K = kc[q];
            ldpc_status st = b_prepare(b, llr, s);
            if (st != LDPC_OK) return st;
            LDPC_CUDA_TRY(cudaEventRecord(e0, s));
            b_loop(b, b->o.max_iter, s);
            LDPC_CUDA_TRY(cudaEventRecord(e1, s));
            LDPC_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            LDPC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            b->tune_k_ms[q] = ms;
            if (ms < kbest) kbest = ms, kb = kc[q];
        }
        b->K = kb;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = true;
    return LDPC_OK;
}

}  // namespace ldpc

extern "C" {

ldpc_status ldpc_batch_decode(ldpc_batch b, const float *const *llr, uint8_t *const *hard, int32_t *const *iters,
                              int32_t *const *ok, void *stream) {
    if (!b || !llr) {
        set_error("need a batch and its llr pointer array");
        return LDPC_EINVAL;
    }
    for (int i = 0; i < b->ncodes; ++i) {
        if (!llr[i] || pointer_kind(llr[i]) != 0 || (hard && hard[i] && pointer_kind(hard[i]) != 0) ||
            (iters && iters[i] && pointer_kind(iters[i]) != 0) || (ok && ok[i] && pointer_kind(ok[i]) != 0)) {
            set_error("code %d: llr (and any outputs) must be device buffers", i);
            return LDPC_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    ldpc_status st;
    if (!b->tuned) {
        st = b_tune(b, llr, s);
        if (st != LDPC_OK) return st;
    }
    st = b_prepare(b, llr, s);
    if (st != LDPC_OK) return st;
    if (!b->exec) {
        // the first run goes eagerly (kernel attributes get set), then the loop is captured
        b_loop(b, b->o.max_iter, s);
        LDPC_CUDA_TRY(cudaGetLastError());
        cudaStream_t cs;
        LDPC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        LDPC_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        b_loop(b, b->o.max_iter, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &b->graph);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        LDPC_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    } else {
        LDPC_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    }
    for (int i = 0; i < b->ncodes; ++i) {
        ldpc_code_s &v = b->views[i];
        const int g = b->hcodes[i].gamma;
        st = qc_finish(&v, g, b->o, s);
        if (st != LDPC_OK) return st;
        st = qc_unpack_outputs(&v, g, b->o, nullptr, hard ? hard[i] : nullptr, iters ? iters[i] : nullptr,
                               ok ? ok[i] : nullptr, s);
        if (st != LDPC_OK) return st;
    }
    if (b->o.early_stop && b->K > 0 && b->K < b->o.max_iter) {
        // frames moved to the second areas: the syndrome of their last decisions, then their rows of
        // the outputs (one launch each over all codes)
        const int nc = b->ncodes;
        LDPC_CUDA_TRY(cudaEventSynchronize(b->ptr_ev));  // the previous decode's copy has read h_ptrs
        for (int i = 0; i < nc; ++i) {
            b->h_ptrs[i] = hard ? (void *)hard[i] : nullptr;
            b->h_ptrs[nc + i] = iters ? (void *)iters[i] : nullptr;
            b->h_ptrs[2 * nc + i] = ok ? (void *)ok[i] : nullptr;
        }
        const size_t pb = (size_t)nc * sizeof(void *);
        LDPC_CUDA_TRY(cudaMemcpyAsync(b->d_hard, b->h_ptrs, pb, cudaMemcpyHostToDevice, s));
        LDPC_CUDA_TRY(cudaMemcpyAsync(b->d_iters, b->h_ptrs + nc, pb, cudaMemcpyHostToDevice, s));
        LDPC_CUDA_TRY(cudaMemcpyAsync(b->d_ok, b->h_ptrs + 2 * nc, pb, cudaMemcpyHostToDevice, s));
        LDPC_CUDA_TRY(cudaEventRecord(b->ptr_ev, s));
        const dim3 grd((unsigned)(b->sms * 2), (unsigned)nc);
        bsec_syndrome_kernel<<<grd, 256, 0, s>>>(b->codes, b->shtab, b->hw, b->flags, b->moved, nc, b->V);
        bscatter_kernel<<<grd, 256, 0, s>>>(b->codes, b->hw, b->flags, b->iters, b->map, b->moved, nc, b->V,
                                            b->o.max_iter, b->d_hard, b->d_iters, b->d_ok);
        count_launch(2);
        LDPC_CUDA_TRY(cudaGetLastError());
    }
    return LDPC_OK;
}

ldpc_status ldpc_batch_set_compaction(ldpc_batch b, int32_t after_iter) {
    if (!b || after_iter < -1) {
        set_error("need a batch and after_iter >= -1");
        return LDPC_EINVAL;
    }
    b->K = after_iter;
    if (after_iter < 0) b->tuned = false;  // tuned again by the next decode
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return LDPC_OK;
}

ldpc_status ldpc_batch_moved(ldpc_batch b, int32_t *moved) {
    if (!b || !moved) {
        set_error("need a batch and moved");
        return LDPC_EINVAL;
    }
    LDPC_CUDA_TRY(cudaMemcpy(moved, b->moved, (size_t)b->ncodes * sizeof(int), cudaMemcpyDeviceToHost));
    return LDPC_OK;
}

ldpc_status ldpc_batch_info(ldpc_batch b, int32_t *tile_rows, int32_t *tile_groups, double *tune_ms3) {
    if (!b) {
        set_error("batch is NULL");
        return LDPC_EINVAL;
    }
    if (tile_rows) *tile_rows = b->TR;
    if (tile_groups) *tile_groups = b->TG;
    if (tune_ms3)
        for (int q = 0; q < 3; ++q) tune_ms3[q] = b->tune_ms[q];
    return LDPC_OK;
}

ldpc_status ldpc_batch_compaction(ldpc_batch b, int32_t *after_iter, double *tune_ms4) {
    if (!b || !after_iter) {
        set_error("need a batch and after_iter");
        return LDPC_EINVAL;
    }
    *after_iter = b->K;
    if (tune_ms4)
        for (int q = 0; q < 4; ++q) tune_ms4[q] = b->tune_k_ms[q];
    return LDPC_OK;
}

}  // extern "C"

// Systematic encoding on the device: the transmitted codewords of the
// simulation (Sec. V makes the codeword on the GPU together with the noise).
//
// Information set: scanning the columns of H from n = N-1 down to 0, column n
// is a parity position when it is not in the GF(2) span of the columns to its
// right.  Gauss-Jordan elimination of [H | I_M] with the columns of H taken in
// that order finds exactly these pivots, and the rows i < rank of the right
// block give T with T H = [rows of the reduced H]: for a codeword c,
//     c[par_pos[i]] = sum_m T[i][m] s[m]   (GF(2)),   s = H_info u,
// u[j] = c[info_pos[j]], H_info the columns of H at the information positions.
// s is sparse work (the edges of the information columns); T is rank x M, so
// the dense part is M / k times smaller than the rank x k generator block.
//
// Device layout.  Frames are processed in groups of 32, bit-sliced: word x of a
// group holds bit x of its 32 frames (bit b = frame b), the form the decoder's
// hard-decision words already take.  Per group the scratch row sl[g][N + M]
// holds the k information words (index j), the rank parity words (k + i) and
// the M syndrome words (N + m).
//   slice:    information bits -> sliced words (32 ballots per 32 bits)
//   syndrome: s_m = XOR of U_j over the information columns of row m
//   parity:   acc_i ^= T[i][m] * s_m over m, four bits at a time through
//             16-entry tables of the XORs of 4 consecutive s_m (the "four
//             Russians" idea), two rows per thread, T read as column-chunk-major
//             words (coalesced); the check range is split over blocks, which
//             meet through atomic XOR
//   pack:     sliced words -> frame-major bits or bytes (32 ballots per 32 bits)
#include "ldpc_internal.cuh"
#include "qc_device.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

struct ldpc_encoder_s {
    int N = 0, M = 0;
    int64_t k = 0;
    int rank = 0;
    std::vector<int32_t> info_pos;  // [k] increasing
    std::vector<int32_t> par_pos;   // [rank] pivot column of reduced row i
    std::vector<uint32_t> Tt;       // [mc4][rpad] word (c, i): bit t = T[i][32c + t]
    std::vector<int32_t> hrp, hj;   // rows of H_info: information indices of row m in hj[hrp[m] .. hrp[m+1])
    int mc = 0, mc4 = 0, kc = 0, rpad = 0, NW = 0;
    size_t ld = 0;                  // scratch words per group: N + M
    // device
    void *dmem = nullptr;
    const uint32_t *d_Tt = nullptr;
    const int *d_hrp = nullptr, *d_hj = nullptr;
    const int *d_src = nullptr;        // [N] scratch index of position n: j (information) or k + i (parity)
    const uint32_t *d_imask = nullptr; // [NW] bit n: information position
    uint32_t *sl = nullptr;            // [groups][ld] sliced words
    size_t sl_groups = 0;
};

namespace ldpc {

namespace {

constexpr int kEncRows = 512;  // parity rows per block (2 per thread)

// where the frames of a launch come from
struct EncSrc {
    int mode;               // 0: bytes [gamma][k]; 1: frame ids first + f; 2: simulation slots (rlist)
    int gamma;              // frames (modes 0 and 1)
    const uint8_t *bytes;   // mode 0
    uint64_t seed, first;   // modes 1, 2
    const int *rlist;       // mode 2: slots that took a new frame, rcount[parity] of them
    const int *rcount;
    int parity;
    const uint64_t *fid;    // mode 2: frame id of each slot
    __device__ int count() const { return mode == 2 ? rcount[parity] : gamma; }
    __device__ uint64_t frame(int f) const { return mode == 2 ? fid[rlist[f]] : first + (uint64_t)f; }
};

// lane t receives the word whose bit b is bit t of lane b's w (a 32 x 32 bit transpose)
__device__ __forceinline__ uint32_t transpose32(uint32_t w, int lane) {
    uint32_t out = 0u;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint32_t x = __ballot_sync(0xffffffffu, (w >> t) & 1u);
        out = lane == t ? x : out;
    }
    return out;
}

// information bits -> sliced words sl[g][j], j < k.  Block (g, y), warp w: chunk c = 8y + w.
// Blocks y = 0 also clear the group's parity words, which the parity pass accumulates.
__global__ void __launch_bounds__(256) enc_slice_kernel(EncSrc src, int64_t k, int kc, int rank,
                                                        uint32_t *__restrict__ sl, size_t ld) {
    const int g = blockIdx.x;
    const int cnt = src.count();
    if (32 * g >= cnt) return;
    if (blockIdx.y == 0)
        for (int i = threadIdx.x; i < rank; i += blockDim.x) sl[(size_t)g * ld + k + i] = 0u;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (c >= kc) return;
    const int f = 32 * g + lane;
    uint32_t w = 0u;
    if (f < cnt) {
        if (src.mode == 0) {
            const uint8_t *b = src.bytes + (size_t)f * (size_t)k + 32 * (size_t)c;
            const int n = (int)std::min<int64_t>(32, k - 32 * (int64_t)c);
            for (int t = 0; t < n; ++t) w |= (uint32_t)(b[t] & 1u) << t;
        } else {
            const uint64_t F = src.frame(f);
            uint32_t o[4];
            philox4x32_10((uint32_t)(c >> 2), (uint32_t)F, (uint32_t)(F >> 32), 1u, (uint32_t)src.seed,
                          (uint32_t)(src.seed >> 32), o);
            w = o[c & 3];
            const int64_t rem = k - 32 * (int64_t)c;
            if (rem < 32) w &= (1u << rem) - 1u;
        }
    }
    const uint32_t x = transpose32(w, lane);
    if (32 * (int64_t)c + lane < k) sl[(size_t)g * ld + 32 * c + lane] = x;
}

// syndrome of the information part, s_m = XOR_j U_j over the information columns of row m.
// Block (g, y): rows 256y .. 256y + 255.
__global__ void __launch_bounds__(256) enc_syndrome_kernel(EncSrc src, const int *__restrict__ hrp,
                                                           const int *__restrict__ hj, int M, int N,
                                                           uint32_t *__restrict__ sl, size_t ld) {
    const int g = blockIdx.x;
    if (32 * g >= src.count()) return;
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= M) return;
    uint32_t *row = sl + (size_t)g * ld;
    uint32_t x = 0u;
    for (int e = hrp[m]; e < hrp[m + 1]; ++e) x ^= row[hj[e]];
    row[N + m] = x;
}

// parity words sl[g][k + i] ^= XOR_m T[i][m] s_m over the stages of block z (128 checks per
// stage).  Block (g, y, z): rows 512y .. 512y + 511, stages z, z + gridDim.z, ...; the partial
// sums of the z-blocks meet in the (cleared) parity words through atomic XOR.
__global__ void __launch_bounds__(256) enc_parity_kernel(EncSrc src, const uint32_t *__restrict__ Tt, int rpad,
                                                         int M, int mc, int N, int64_t k, int rank,
                                                         uint32_t *__restrict__ sl, size_t ld) {
    __shared__ uint32_t tab[2][32][16];
    const int g = blockIdx.x;
    if (32 * g >= src.count()) return;
    const int tid = threadIdx.x;
    const int r0 = blockIdx.y * kEncRows + tid, r1 = r0 + 256;
    const uint32_t *S = sl + (size_t)g * ld + N;
    uint32_t acc0 = 0u, acc1 = 0u;
    const int ns = (mc + 3) / 4;
    int buf = 0;
    for (int st = blockIdx.z; st < ns; st += gridDim.z, buf ^= 1) {
        // this stage's words of T first: their latency overlaps the table build and the barrier
        uint32_t a0[4], a1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // chunks past mc are zero (the table is padded to mc4)
            a0[q] = __ldg(Tt + (size_t)(4 * st + q) * rpad + r0);
            a1[q] = __ldg(Tt + (size_t)(4 * st + q) * rpad + r1);
        }
        uint32_t(*T)[16] = tab[buf];
        // entry (t, v) = XOR of s_m, m = 128 st + 4 t + b over the set bits b of v
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + 256 * h;
            const int t = e >> 4, v = e & 15;
            uint32_t x = 0u;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int m = 128 * st + 4 * t + b;
                if (((v >> b) & 1) && m < M) x ^= S[m];
            }
            T[t][v] = x;
        }
        // the other table is free: every thread has passed the previous barrier, so the
        // stage that read it is done
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                acc0 ^= T[8 * q + t][(a0[q] >> (4 * t)) & 15u];
                acc1 ^= T[8 * q + t][(a1[q] >> (4 * t)) & 15u];
            }
    }
    if (r0 < rank && acc0) atomicXor(sl + (size_t)g * ld + k + r0, acc0);
    if (r1 < rank && acc1) atomicXor(sl + (size_t)g * ld + k + r1, acc1);
}

// where a pack writes
struct EncDst {
    int mode;           // 0: bytes [gamma][len]; 2: frame-major words cwf[slot][NW]
    uint8_t *bytes;
    uint32_t *cwf;
    int NW;
};

// sliced words -> per-frame bits.  Positions x < len: codeword positions (src != NULL,
// word sl[g][src[x]]) or information bits (src == NULL, word sl[g][x]).
__global__ void __launch_bounds__(256) enc_pack_kernel(EncSrc fs, const uint32_t *__restrict__ sl, size_t ld,
                                                       const int *__restrict__ srcidx, int len, EncDst dst) {
    const int g = blockIdx.x;
    const int cnt = fs.count();
    if (32 * g >= cnt) return;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (32 * c >= len) return;
    const int x = 32 * c + lane;
    uint32_t w = 0u;
    if (x < len) w = sl[(size_t)g * ld + (srcidx ? srcidx[x] : x)];
    const uint32_t bits = transpose32(w, lane);  // lane b: positions 32c .. 32c+31 of frame b
    const int f = 32 * g + lane;
    if (f >= cnt) return;
    if (dst.mode == 2) {
        dst.cwf[(size_t)fs.rlist[f] * dst.NW + c] = bits;
    } else {
        uint8_t *o = dst.bytes + (size_t)f * len + 32 * (size_t)c;
        const int n = len - 32 * c < 32 ? len - 32 * c : 32;
        for (int t = 0; t < n; ++t) o[t] = (uint8_t)((bits >> t) & 1u);
    }
}

// wrong information bits of the frames retiring in package word (pk, v): their decisions
// are the staged hard words hw[pk][n][v] (bit = lane), their codewords the rows cwf[slot].
// Lane L holds the word of variable 32c + L; for each retiring lane b one ballot of bit b
// gives that frame's decisions at 32c .. 32c+31.
template <int V>
__global__ void __launch_bounds__(256) enc_errors_kernel(const uint32_t *__restrict__ hw,
                                                         const uint32_t *__restrict__ sflags,
                                                         const uint32_t *__restrict__ cwf,
                                                         const uint32_t *__restrict__ imask, int *__restrict__ errs,
                                                         int N, int NW) {
    const int pk = blockIdx.x / V, v = blockIdx.x - (blockIdx.x / V) * V;
    const uint32_t ret = sflags[(size_t)pk * 2 * V + v];
    if (!ret) return;
    const int lane = threadIdx.x & 31;
    const bool mine = (ret >> lane) & 1u;
    const size_t slot = (size_t)pk * 32 * V + (size_t)lane * V + v;
    int cnt = 0;
    const int stride = gridDim.y * 8;
    // four chunks per round: their loads are issued together
    for (int c0 = blockIdx.y * 8 + (threadIdx.x >> 5); c0 < NW; c0 += 4 * stride) {
        uint32_t h[4], w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c0 + i * stride, n = 32 * c + lane;
            h[i] = c < NW && n < N ? hw[((size_t)pk * N + n) * V + v] : 0u;
            w[i] = c < NW && mine ? cwf[slot * NW + c] & imask[c] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c0 + i * stride;
            const uint32_t m = c < NW ? imask[c] : 0u;
            uint32_t mydec = 0u;
            for (uint32_t r = ret; r; r &= r - 1) {  // warp-uniform loop over the retiring lanes
                const int b = __ffs(r) - 1;
                const uint32_t d = __ballot_sync(0xffffffffu, (h[i] >> b) & 1u);
                mydec = lane == b ? d : mydec;
            }
            cnt += __popc((mydec & m) ^ w[i]);
        }
    }
    if (mine && cnt) atomicAdd(errs + slot, cnt);
}

// channel LLRs of given codewords (bytes [gamma][N]); as channel_frames_kernel otherwise
__global__ void channel_cw_kernel(float *__restrict__ out, const uint8_t *__restrict__ cw, int N, int gamma,
                                  uint64_t seed, uint64_t first_frame, float sigma, float s2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * q >= N) return;
    for (int f = blockIdx.y; f < gamma; f += gridDim.y) {
        uint32_t bits = 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < N) bits |= (uint32_t)(cw[(size_t)f * N + 4 * q + e] & 1u) << e;
        float v4[4];
        channel_quad(seed, first_frame + (uint64_t)f, q, sigma, s2, v4, bits);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < N) out[(size_t)f * N + 4 * q + e] = v4[e];
    }
}

// H as bit rows [M][W] (W = ceil(N / 64) words)
void parity_rows(const ldpc_code c, std::vector<uint64_t> &R, int W) {
    const int M = c->d.M;
    R.assign((size_t)M * W, 0ull);
    auto set = [&](int m, int n) { R[(size_t)m * W + (n >> 6)] |= 1ull << (n & 63); };
    if (c->sparse) {
        for (int m = 0; m < M; ++m)
            for (int e = c->h_rp[m]; e < c->h_rp[m + 1]; ++e) set(m, c->h_col[e]);
    } else {
        const QcDesc &d = c->d;
        for (int j = 0; j < d.J; ++j)
            for (int l = 0; l < d.L; ++l) {
                const int a = d.shift[j * d.L + l];
                if (a < 0) continue;
                for (int r = 0; r < d.p; ++r) set(j * d.p + r, l * d.p + (r + a) % d.p);
            }
    }
}

ldpc_status launch_encode(ldpc_code c, const EncSrc &src, int groups, cudaStream_t s) {
    ldpc_encoder_s *e = c->enc;
    if (e->kc == 0) {
        // k = 0: the only codeword is zero
        LDPC_CUDA_TRY(cudaMemsetAsync(e->sl, 0, (size_t)groups * e->ld * 4, s));
        return LDPC_OK;
    }
    enc_slice_kernel<<<dim3(groups, (e->kc + 7) / 8), 256, 0, s>>>(src, e->k, e->kc, e->rank, e->sl, e->ld);
    count_launch();
    if (e->rank > 0) {
        enc_syndrome_kernel<<<dim3(groups, (e->M + 255) / 256), 256, 0, s>>>(src, e->d_hrp, e->d_hj, e->M, e->N,
                                                                            e->sl, e->ld);
        // split the stages so that each block runs about 4 of them
        const int ns = (e->mc + 3) / 4, zs = std::min(16, (ns + 3) / 4);
        enc_parity_kernel<<<dim3(groups, e->rpad / kEncRows, zs), 256, 0, s>>>(
            src, e->d_Tt, e->rpad, e->M, e->mc, e->N, e->k, e->rank, e->sl, e->ld);
        count_launch(2);
    }
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status launch_pack(ldpc_code c, const EncSrc &src, int groups, const int *srcidx, int len, const EncDst &dst,
                        cudaStream_t s) {
    if (len <= 0) return LDPC_OK;
    const int chunks = (len + 31) / 32;
    enc_pack_kernel<<<dim3(groups, (chunks + 7) / 8), 256, 0, s>>>(src, c->enc->sl, c->enc->ld, srcidx, len, dst);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace

void enc_free(ldpc_encoder_s *e) {
    if (!e) return;
    cudaFree(e->dmem);
    cudaFree(e->sl);
    delete e;
}

int64_t enc_k(const ldpc_code c) { return c->enc ? c->enc->k : -1; }
int enc_words(const ldpc_code c) { return (c->d.N + 31) / 32; }

ldpc_status enc_build_host(ldpc_code c) {
    std::lock_guard<std::mutex> lock(c->enc_mu);
    if (c->enc) return LDPC_OK;
    const int M = c->d.M, N = c->d.N, W = (N + 63) / 64;
    std::vector<uint64_t> H0;
    parity_rows(c, H0, W);
    // [H | I_M] by rows, W2 words each
    const int W2 = (N + M + 63) / 64;
    std::vector<uint64_t> R((size_t)M * W2, 0ull);
    for (int m = 0; m < M; ++m) {
        std::copy(H0.begin() + (size_t)m * W, H0.begin() + (size_t)(m + 1) * W, R.begin() + (size_t)m * W2);
        const int b = N + m;
        R[(size_t)m * W2 + (b >> 6)] |= 1ull << (b & 63);
    }
    // Gauss-Jordan over GF(2), pivot columns taken from n = N-1 down to 0
    std::vector<int32_t> piv;
    int rank = 0;
    for (int n = N - 1; n >= 0 && rank < M; --n) {
        const int w = n >> 6;
        const uint64_t b = 1ull << (n & 63);
        int r = rank;
        while (r < M && !(R[(size_t)r * W2 + w] & b)) ++r;
        if (r == M) continue;
        if (r != rank) std::swap_ranges(R.begin() + (size_t)r * W2, R.begin() + (size_t)(r + 1) * W2,
                                        R.begin() + (size_t)rank * W2);
        const uint64_t *pr = R.data() + (size_t)rank * W2;
        for (int q = 0; q < M; ++q) {
            if (q == rank) continue;
            uint64_t *x = R.data() + (size_t)q * W2;
            if (x[w] & b)
                for (int t = 0; t < W2; ++t) x[t] ^= pr[t];
        }
        piv.push_back(n);
        ++rank;
    }
    ldpc_encoder_s *e = new (std::nothrow) ldpc_encoder_s();
    if (!e) {
        set_error("host allocation failed");
        return LDPC_ENOMEM;
    }
    e->N = N;
    e->M = M;
    e->rank = rank;
    e->par_pos = piv;
    std::vector<int> idx(N, -1);  // information index of column n, -1 for a pivot column
    for (int i = 0; i < rank; ++i) idx[piv[i]] = -2;
    for (int n = 0; n < N; ++n)
        if (idx[n] == -1) {
            idx[n] = (int)e->info_pos.size();
            e->info_pos.push_back(n);
        } else {
            idx[n] = -1;
        }
    e->k = (int64_t)e->info_pos.size();
    e->kc = (int)((e->k + 31) / 32);
    e->mc = (M + 31) / 32;
    e->mc4 = (e->mc + 3) / 4 * 4;
    e->rpad = (rank + kEncRows - 1) / kEncRows * kEncRows;
    e->NW = (N + 31) / 32;
    e->ld = (size_t)N + (size_t)M;
    // T: the identity block of the reduced rows, column-chunk-major
    e->Tt.assign((size_t)e->mc4 * e->rpad, 0u);
    for (int i = 0; i < rank; ++i) {
        const uint64_t *row = R.data() + (size_t)i * W2;
        for (int m = 0; m < M; ++m) {
            const int bit = N + m;
            if ((row[bit >> 6] >> (bit & 63)) & 1ull) e->Tt[(size_t)(m >> 5) * e->rpad + i] |= 1u << (m & 31);
        }
    }
    // H_info by rows
    e->hrp.assign(M + 1, 0);
    for (int m = 0; m < M; ++m) {
        const uint64_t *row = H0.data() + (size_t)m * W;
        for (int w = 0; w < W; ++w) {
            uint64_t x = row[w];
            while (x) {
                const int n = 64 * w + __builtin_ctzll(x);
                x &= x - 1;
                if (idx[n] >= 0) e->hj.push_back(idx[n]);
            }
        }
        e->hrp[m + 1] = (int)e->hj.size();
    }
    c->enc = e;
    return LDPC_OK;
}

ldpc_status enc_ensure_device(ldpc_code c, size_t groups) {
    ldpc_status st = enc_build_host(c);
    if (st != LDPC_OK) return st;
    std::lock_guard<std::mutex> lock(c->enc_mu);
    ldpc_encoder_s *e = c->enc;
    const int N = e->N, M = e->M;
    if (!e->dmem) {
        const size_t nt = e->Tt.size(), nj = e->hj.size();
        const size_t words = nt + (size_t)(M + 1) + nj + (size_t)N + (size_t)e->NW;
        void *mem = nullptr;
        if (cudaMalloc(&mem, words * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of the encoder tables (%zu bytes) failed", words * 4);
            return LDPC_ENOMEM;
        }
        std::vector<int> src(N);
        std::vector<uint32_t> imask(e->NW, 0u);
        for (int64_t j = 0; j < e->k; ++j) {
            const int n = e->info_pos[(size_t)j];
            src[n] = (int)j;
            imask[n >> 5] |= 1u << (n & 31);
        }
        for (int i = 0; i < e->rank; ++i) src[e->par_pos[i]] = (int)(e->k + i);
        uint32_t *base = (uint32_t *)mem;
        uint32_t *p_hrp = base + nt, *p_hj = p_hrp + M + 1, *p_src = p_hj + nj, *p_im = p_src + N;
        cudaError_t ce = cudaMemcpy(base, e->Tt.data(), nt * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(p_hrp, e->hrp.data(), (size_t)(M + 1) * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess && nj) ce = cudaMemcpy(p_hj, e->hj.data(), nj * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(p_src, src.data(), (size_t)N * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(p_im, imask.data(), (size_t)e->NW * 4, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            cudaFree(mem);
            return cuda_fail(ce, "cudaMemcpy(encoder tables)");
        }
        e->dmem = mem;
        e->d_Tt = base;
        e->d_hrp = (const int *)p_hrp;
        e->d_hj = (const int *)p_hj;
        e->d_src = (const int *)p_src;
        e->d_imask = p_im;
    }
    if (groups > e->sl_groups) {
        LDPC_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(e->sl);
        e->sl = nullptr;
        e->sl_groups = 0;
        if (cudaMalloc(&e->sl, groups * e->ld * 4) != cudaSuccess) {
            cudaGetLastError();
            e->sl = nullptr;
            set_error("device allocation of the encoder scratch (%zu groups) failed", groups);
            return LDPC_ENOMEM;
        }
        e->sl_groups = groups;
    }
    return LDPC_OK;
}

ldpc_status enc_sim_errors(ldpc_code c, int P, int V, const uint32_t *sflags, const uint32_t *cwf, int *errs,
                           cudaStream_t s) {
    const ldpc_encoder_s *e = c->enc;
    const dim3 grd(P * V, std::min(8, (e->NW + 7) / 8));
    if (V == 1) enc_errors_kernel<1><<<grd, 256, 0, s>>>(c->ws.hw, sflags, cwf, e->d_imask, errs, e->N, e->NW);
    else if (V == 2) enc_errors_kernel<2><<<grd, 256, 0, s>>>(c->ws.hw, sflags, cwf, e->d_imask, errs, e->N, e->NW);
    else enc_errors_kernel<4><<<grd, 256, 0, s>>>(c->ws.hw, sflags, cwf, e->d_imask, errs, e->N, e->NW);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status enc_sim_codewords(ldpc_code c, int slots, const int *rlist, const int *rcount, int parity,
                              const uint64_t *fid, uint64_t seed, uint32_t *cwf, cudaStream_t s) {
    EncSrc src{};
    src.mode = 2;
    src.seed = seed;
    src.rlist = rlist;
    src.rcount = rcount;
    src.parity = parity;
    src.fid = fid;
    const int groups = (slots + 31) / 32;
    ldpc_status st = launch_encode(c, src, groups, s);
    if (st != LDPC_OK) return st;
    EncDst dst{};
    dst.mode = 2;
    dst.cwf = cwf;
    dst.NW = c->enc->NW;
    return launch_pack(c, src, groups, c->enc->d_src, c->enc->N, dst, s);
}

}  // namespace ldpc

using namespace ldpc;

namespace {

// frames per pass of the device-buffer calls (bounds the sliced scratch)
constexpr int kEncChunk = 4096;

ldpc_status check_device(const void *p, const char *what) {
    if (p && pointer_kind(p) != 0) {
        set_error("%s must be a device pointer", what);
        return LDPC_EINVAL;
    }
    return LDPC_OK;
}

ldpc_status encode_frames(ldpc_code c, int mode, const uint8_t *info_in, uint64_t seed, uint64_t first, int gamma,
                          uint8_t *info_out, uint8_t *cw, cudaStream_t s) {
    ldpc_status st = enc_ensure_device(c, (size_t)(std::min(gamma, kEncChunk) + 31) / 32);
    if (st != LDPC_OK) return st;
    ldpc_encoder_s *e = c->enc;
    for (int f0 = 0; f0 < gamma; f0 += kEncChunk) {
        const int n = std::min(kEncChunk, gamma - f0);
        const int groups = (n + 31) / 32;
        EncSrc src{};
        src.mode = mode;
        src.gamma = n;
        src.bytes = info_in ? info_in + (size_t)f0 * (size_t)e->k : nullptr;
        src.seed = seed;
        src.first = first + (uint64_t)f0;
        st = launch_encode(c, src, groups, s);
        if (st != LDPC_OK) return st;
        EncDst dst{};
        dst.mode = 0;
        dst.bytes = cw + (size_t)f0 * e->N;
        st = launch_pack(c, src, groups, e->d_src, e->N, dst, s);
        if (st != LDPC_OK) return st;
        if (info_out) {
            dst.bytes = info_out + (size_t)f0 * (size_t)e->k;
            st = launch_pack(c, src, groups, nullptr, (int)e->k, dst, s);
            if (st != LDPC_OK) return st;
        }
    }
    return LDPC_OK;
}

}  // namespace

extern "C" {

ldpc_status ldpc_code_info_set(ldpc_code c, int64_t *k, int32_t *info_pos) {
    if (!c) {
        set_error("code is NULL");
        return LDPC_EINVAL;
    }
    ldpc_status st = enc_build_host(c);
    if (st != LDPC_OK) return st;
    if (k) *k = c->enc->k;
    if (info_pos && c->enc->k > 0) std::memcpy(info_pos, c->enc->info_pos.data(), (size_t)c->enc->k * 4);
    return LDPC_OK;
}

ldpc_status ldpc_encode(ldpc_code c, const uint8_t *info, int32_t gamma, uint8_t *cw, void *stream) {
    if (!c || !cw || gamma < 1) {
        set_error("need code, cw and gamma >= 1");
        return LDPC_EINVAL;
    }
    ldpc_status st = enc_build_host(c);
    if (st != LDPC_OK) return st;
    if (!info && c->enc->k > 0) {
        set_error("info is NULL but k = %lld", (long long)c->enc->k);
        return LDPC_EINVAL;
    }
    if ((st = check_device(info, "info")) != LDPC_OK || (st = check_device(cw, "cw")) != LDPC_OK) return st;
    return encode_frames(c, 0, info, 0, 0, gamma, nullptr, cw, (cudaStream_t)stream);
}

ldpc_status ldpc_random_codewords(ldpc_code c, uint64_t seed, uint64_t first_frame, int32_t gamma, uint8_t *info,
                                  uint8_t *cw, void *stream) {
    if (!c || !cw || gamma < 1) {
        set_error("need code, cw and gamma >= 1");
        return LDPC_EINVAL;
    }
    ldpc_status st;
    if ((st = check_device(info, "info")) != LDPC_OK || (st = check_device(cw, "cw")) != LDPC_OK) return st;
    return encode_frames(c, 1, nullptr, seed, first_frame, gamma, info, cw, (cudaStream_t)stream);
}

ldpc_status ldpc_channel_codewords(ldpc_code c, double ebn0_db, uint64_t seed, uint64_t first_frame, int32_t gamma,
                                   const uint8_t *cw, float *llr_out, void *stream) {
    if (!c || !cw || !llr_out || gamma < 1 || !std::isfinite(ebn0_db)) {
        set_error("need code, cw, llr_out, gamma >= 1 and a finite Eb/N0");
        return LDPC_EINVAL;
    }
    if (!(c->rate > 0.0)) {
        set_error("design rate K/N = %g is not positive", c->rate);
        return LDPC_EINVAL;
    }
    ldpc_status st;
    if ((st = check_device(cw, "cw")) != LDPC_OK || (st = check_device(llr_out, "llr_out")) != LDPC_OK) return st;
    const double sigma = channel_sigma(c, ebn0_db);
    const int N = c->d.N;
    const dim3 grd(((N + 3) / 4 + 127) / 128, std::min(gamma, 65535));
    channel_cw_kernel<<<grd, 128, 0, (cudaStream_t)stream>>>(llr_out, cw, N, gamma, seed, first_frame, (float)sigma,
                                                             (float)(2.0 / (sigma * sigma)));
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"

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

#include <cmath>
#include <new>
#include <numeric>
#include <vector>

struct ldpccc_s {
    ldpc::QcDesc d;          // base code
    int lam, Jb, Lb, c, cb, ms, I, gamma, P, ring;
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

// check pass of slot t over the I processors' layers; one warp = one check row of one package
template <int DCMAX>
__global__ void __launch_bounds__(kWarps * 32)
cc_cn_kernel(const QcDesc d, CcDesc g, uint32_t *__restrict__ msg, const float *__restrict__ mu, long long t,
             float clip) {
    const int lane = threadIdx.x & 31;
    const int row_all = blockIdx.x * kWarps + (threadIdx.x >> 5);  // over I * cb
    const int pk = blockIdx.y;
    if (row_all >= g.I * g.cb) return;
    const int i = row_all / g.cb, row = row_all - i * g.cb;
    const long long R = t - (long long)i * g.lam;
    if (R < 0) return;
    const int a = mod_pos(R, g.lam);
    const int jj = row / d.p, r = row - jj * d.p;
    const int j = a * g.Jb + jj;
    const bool proc1 = i == 0;
    float ph[DCMAX];
    size_t addr[DCMAX];
    uint32_t neg = 0u;
#pragma unroll
    for (int l = 0; l < DCMAX; ++l) {
        ph[l] = 0.0f;
        addr[l] = ~(size_t)0;
        if (l >= d.L) continue;
        const int sh = d.shift[j * d.L + l];
        if (sh < 0) continue;
        const int b = l / g.Lb, ll = l - b * g.Lb;
        const long long F = R - mod_pos(a - b, g.lam);
        if (F < 0) continue;
        int k = r + sh;
        if (k >= d.p) k -= d.p;
        const int slot = mod_pos(F, g.ring);
        const size_t e = (size_t)(j * g.Lb + ll) * d.p + k;
        addr[l] = (((size_t)slot * g.P + pk) * g.Ef + e) * 32 + lane;
        float x;
        if (proc1) {
            x = mu[(((size_t)slot * g.P + pk) * g.c + (size_t)ll * d.p + k) * 32 + lane];
            ph[l] = phi_f(fabsf(x));
        } else {
            x = __uint_as_float(msg[addr[l]]);
            ph[l] = fabsf(x);  // the variable pass stored sign(beta) * phi(|beta|)
        }
        neg |= (x < 0.0f ? 1u : 0u) << l;
    }
    float pre[DCMAX];
    float acc = 0.0f;
#pragma unroll
    for (int l = 0; l < DCMAX; ++l) {
        pre[l] = acc;
        acc += ph[l];
    }
    const uint32_t par = __popc(neg) & 1u;
    float suf = 0.0f;
#pragma unroll
    for (int l = DCMAX - 1; l >= 0; --l) {
        if (addr[l] != ~(size_t)0) {
            const float mag = fminf(phi_f(pre[l] + suf), clip);
            msg[addr[l]] = __float_as_uint((par ^ ((neg >> l) & 1u)) ? -mag : mag);
        }
        suf += ph[l];
    }
}

// variable pass of slot t over the I processors' frames; one warp = one variable of one package.
// The frame leaving processor I gets its posterior and hard decision (output index q).
template <int JMAX>
__global__ void __launch_bounds__(kWarps * 32)
cc_vn_kernel(const QcDesc d, CcDesc g, uint32_t *__restrict__ msg, const float *__restrict__ mu, long long t,
             float clip, int gamma, int T_out, int q_out, uint8_t *__restrict__ hard, float *__restrict__ post) {
    const int lane = threadIdx.x & 31;
    const int var_all = blockIdx.x * kWarps + (threadIdx.x >> 5);  // over I * c
    const int pk = blockIdx.y;
    if (var_all >= g.I * g.c) return;
    const int i = var_all / g.c, v = var_all - i * g.c;
    const long long F = t - (long long)i * g.lam - g.ms;
    if (F < 0) return;
    const int b = mod_pos(F, g.lam);
    const int slot = mod_pos(F, g.ring);
    const int ll = v / d.p, k = v - ll * d.p;
    const int l = b * g.Lb + ll;
    const float m = mu[(((size_t)slot * g.P + pk) * g.c + v) * 32 + lane];
    float a[JMAX];
    size_t addr[JMAX];
    float tot = m;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        a[j] = 0.0f;
        addr[j] = ~(size_t)0;
        if (j >= d.J || d.shift[j * d.L + l] < 0) continue;
        const size_t e = (size_t)(j * g.Lb + ll) * d.p + k;
        addr[j] = (((size_t)slot * g.P + pk) * g.Ef + e) * 32 + lane;
        a[j] = __uint_as_float(msg[addr[j]]);
        tot += a[j];
    }
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        if (addr[j] == ~(size_t)0) continue;
        float s = m;
#pragma unroll
        for (int j2 = 0; j2 < JMAX; ++j2)
            if (j2 != j) s += a[j2];
        const float bt = clipf(s, clip);
        const float f = phi_f(fabsf(bt));
        msg[addr[j]] = __float_as_uint(bt < 0.0f ? -f : f);
    }
    if (i == g.I - 1 && q_out >= 0) {
        const float pst = clipf(tot, clip);
        const int s = pk * 32 + lane;
        if (s < gamma) {
            const size_t o = ((size_t)s * T_out + q_out) * g.c + v;
            if (hard) hard[o] = pst < 0.0f ? 1 : 0;
            if (post) post[o] = pst;
        }
    }
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
    return CcDesc{cc->lam, cc->Jb, cc->Lb, cc->c, cc->cb, cc->ms, cc->I, cc->P, cc->ring, cc->d.J * cc->c};
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpccc_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                          ldpccc *out) {
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
    cc->lam = std::gcd(J, L);
    cc->Jb = J / cc->lam;
    cc->Lb = L / cc->lam;
    cc->c = cc->Lb * p;
    cc->cb = cc->Jb * p;
    cc->ms = cc->lam - 1;
    cc->I = I;
    cc->gamma = gamma;
    cc->P = (gamma + 31) / 32;
    cc->ring = I * cc->lam;
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
    if (lambda) *lambda = cc->lam;
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
    dim3 cgrd((cc->I * cc->cb + kWarps - 1) / kWarps, cc->P);
    dim3 vgrd((cc->I * cc->c + kWarps - 1) / kWarps, cc->P);
    for (int tt = 0; tt < T; ++tt) {
        const long long t = t0 + tt;
        cc_enter_kernel<<<egrd, eblk, 0, s>>>(src, cc->mu, g, cc->gamma, T, tt, t, clip);
        if (dcm <= 8) cc_cn_kernel<8><<<cgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip);
        else if (dcm <= 16) cc_cn_kernel<16><<<cgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip);
        else if (dcm <= 24) cc_cn_kernel<24><<<cgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip);
        else cc_cn_kernel<32><<<cgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip);
        const long long Fd = t - (long long)cc->ring + 1;  // frame decided at this slot
        const int q = Fd >= 0 ? (int)(Fd - (first_dec > 0 ? first_dec : 0)) : -1;
        if (q >= 0) ++n;
        if (cc->d.J <= 4)
            cc_vn_kernel<4><<<vgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip, cc->gamma, T, q, dh, dp);
        else
            cc_vn_kernel<8><<<vgrd, kWarps * 32, 0, s>>>(cc->d, g, cc->msg, cc->mu, t, clip, cc->gamma, T, q, dh, dp);
        count_launch(3);
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

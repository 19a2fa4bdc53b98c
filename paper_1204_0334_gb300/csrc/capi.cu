// C-ABI entry points of the block-code decoder (include/ldpc.h).
#include "ldpc_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace ldpc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ldpc_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return LDPC_ECUDA;
}

double channel_sigma(const ldpc_code c, double ebn0_db) {
    return std::sqrt(1.0 / (2.0 * c->rate * std::pow(10.0, ebn0_db / 10.0)));
}

int pointer_kind(const void *p) {
    if (!p) return -1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 0 : 1;
}

ldpc_status check_opts(const ldpc_code c, const ldpc_decode_opts *o) {
    if (!o) {
        set_error("opts is NULL");
        return LDPC_EINVAL;
    }
    if (o->max_iter < 1 || o->max_iter > 100000) {
        set_error("max_iter %d out of range [1, 100000]", o->max_iter);
        return LDPC_EINVAL;
    }
    if (c && c->sparse && o->algo == LDPC_ALGO_NOMS) {
        set_error("the learned min-sum takes QC codes (parameters per circulant)");
        return LDPC_EUNSUPPORTED;
    }
    if (o->codewords != LDPC_CODEWORDS_ZERO && o->codewords != LDPC_CODEWORDS_RANDOM) {
        set_error("codewords must be LDPC_CODEWORDS_ZERO or LDPC_CODEWORDS_RANDOM (got %d)", o->codewords);
        return LDPC_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (o->reserved[i]) {
            set_error("reserved fields must be zero");
            return LDPC_EINVAL;
        }
    if (o->algo == LDPC_ALGO_SP) {
        if (o->msg != LDPC_MSG_F32 && o->msg != LDPC_MSG_F16) {
            set_error("sum-product takes F32 or F16 messages");
            return LDPC_EUNSUPPORTED;
        }
        if (!(o->clip > 0.0f) || !std::isfinite(o->clip) || o->clip > 60000.0f) {
            set_error("clip must be finite, positive and representable in FP16 storage");
            return LDPC_EINVAL;
        }
    } else if (o->algo == LDPC_ALGO_MS) {
        if (o->msg != LDPC_MSG_I8) {
            set_error("integer min-sum takes I8 messages");
            return LDPC_EUNSUPPORTED;
        }
        if (o->frac_bits < 0 || o->frac_bits > 6) {
            set_error("frac_bits %d out of range [0, 6]", o->frac_bits);
            return LDPC_EINVAL;
        }
    } else if (o->algo == LDPC_ALGO_NOMS) {
        if (o->msg != LDPC_MSG_F32 && o->msg != LDPC_MSG_F16) {
            set_error("normalized/offset min-sum takes F32 or F16 messages");
            return LDPC_EUNSUPPORTED;
        }
        if (!o->noms_params || pointer_kind(o->noms_params) != 0 || ((uintptr_t)o->noms_params & 7u)) {
            set_error("NOMS needs device noms_params [max_iter][J*L][2], 8-byte aligned");
            return LDPC_EINVAL;
        }
        if (!(o->clip > 0.0f) || !std::isfinite(o->clip) || o->clip > 60000.0f) {
            set_error("clip must be finite, positive and representable in FP16 storage");
            return LDPC_EINVAL;
        }
    } else {
        set_error("unknown algo %d", o->algo);
        return LDPC_EINVAL;
    }
    (void)c;
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

void ldpc_default_opts(ldpc_decode_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->max_iter = 30;
    o->early_stop = 0;
    o->algo = LDPC_ALGO_SP;
    o->msg = LDPC_MSG_F32;
    o->clip = 30.0f;
    o->frac_bits = 2;
}

const char *ldpc_status_str(ldpc_status s) {
    switch (s) {
        case LDPC_OK: return "ok";
        case LDPC_EINVAL: return "invalid argument";
        case LDPC_ENOMEM: return "out of memory";
        case LDPC_ECUDA: return "CUDA error";
        case LDPC_ETIMEOUT: return "device wait timed out";
        case LDPC_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *ldpc_last_error(void) { return g_err; }

ldpc_status ldpc_code_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, ldpc_code *out) {
    if (!out) {
        set_error("out is NULL");
        return LDPC_EINVAL;
    }
    *out = nullptr;
    if (!shifts || J < 1 || J > kMaxJ || L < 1 || L > kMaxL || p < 1) {
        set_error("need shifts != NULL, 1 <= J <= %d, 1 <= L <= %d, p >= 1 (got J=%d L=%d p=%d)", kMaxJ, kMaxL, J, L,
                  p);
        return LDPC_EINVAL;
    }
    if ((int64_t)L * p > (1 << 26)) {
        set_error("code too long: N = %lld", (long long)L * p);
        return LDPC_EINVAL;
    }
    QcDesc d;
    std::memset(&d, 0, sizeof(d));
    d.J = J;
    d.L = L;
    d.p = p;
    d.N = L * p;
    d.M = J * p;
    int e = 0, dcmax = 0;
    for (int j = 0; j < kMaxJ * kMaxL; ++j) d.shift[j] = -1, d.eoff[j] = -1;
    for (int j = 0; j < J; ++j) {
        int dc = 0;
        for (int l = 0; l < L; ++l) {
            const int a = shifts[j * L + l];
            if (a < -1 || a >= p) {
                set_error("shift a[%d][%d] = %d outside {-1} u [0, %d)", j, l, a, p);
                return LDPC_EINVAL;
            }
            d.shift[j * L + l] = a;
            if (a >= 0) {
                d.eoff[j * L + l] = e;
                e += p;
                ++dc;
            }
        }
        dcmax = dc > dcmax ? dc : dcmax;
    }
    d.E = e;
    // the kernels index by the block column, so the row degree bound is L
    d.dc_max = L;
    d.divM = fast_div((uint32_t)d.M);
    d.divP = fast_div((uint32_t)d.p);
    d.divG = fast_div((uint32_t)((d.N + 3) / 4));
    (void)dcmax;
    ldpc_code c = new (std::nothrow) ldpc_code_s();
    if (!c) {
        set_error("host allocation failed");
        return LDPC_ENOMEM;
    }
    c->d = d;
    c->rate = 1.0 - (double)d.M / (double)d.N;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        c->device = 0;
    }
    *out = c;
    return LDPC_OK;
}

ldpc_status ldpc_code_destroy(ldpc_code c) {
    if (!c) return LDPC_OK;
    DecodeWs &w = c->ws;
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
    noms_free(c->noms);
    sim_free(c->sim);
    enc_free(c->enc);
    cudaFree(c->sp_mem);
    delete c;
    return LDPC_OK;
}

ldpc_status ldpc_code_create_sparse(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                                    ldpc_code *out) {
    if (!out || !row_ptr || !col_idx || M < 1 || N < 1) {
        set_error("need out, row_ptr, col_idx, M >= 1 and N >= 1");
        return LDPC_EINVAL;
    }
    *out = nullptr;
    if (row_ptr[0] != 0) {
        set_error("row_ptr[0] = %d, expected 0", row_ptr[0]);
        return LDPC_EINVAL;
    }
    int dc_max = 0;
    for (int m = 0; m < M; ++m) {
        const int a = row_ptr[m], b = row_ptr[m + 1];
        if (b - a < 1 || b - a > 32) {
            set_error("row %d has degree %d outside [1, 32]", m, b - a);
            return LDPC_EINVAL;
        }
        dc_max = std::max(dc_max, b - a);
        for (int e = a; e < b; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= N || (e > a && col_idx[e] <= col_idx[e - 1])) {
                set_error("row %d: column indices must increase within [0, %d)", m, N);
                return LDPC_EINVAL;
            }
        }
    }
    const long long E = row_ptr[M];
    if (E * 32 >= (1ll << 31)) {
        set_error("E = %lld edges: E * 32 must stay below 2^31", E);
        return LDPC_EINVAL;
    }
    // each variable's edges (rows increase because edges are numbered row by row)
    std::vector<int> cptr(N + 1, 0), cedge((size_t)E);
    for (long long e = 0; e < E; ++e) ++cptr[col_idx[e] + 1];
    int dv_max = 0;
    for (int n = 0; n < N; ++n) {
        dv_max = std::max(dv_max, cptr[n + 1]);
        cptr[n + 1] += cptr[n];
    }
    if (dv_max > 8) {
        set_error("a column has degree %d > 8", dv_max);
        return LDPC_EINVAL;
    }
    {
        std::vector<int> fill(cptr.begin(), cptr.end() - 1);
        for (long long e = 0; e < E; ++e) cedge[(size_t)fill[col_idx[e]]++] = (int)e;
    }
    ldpc_code c = new (std::nothrow) ldpc_code_s();
    if (!c) {
        set_error("host allocation failed");
        return LDPC_ENOMEM;
    }
    std::memset(&c->d, 0, sizeof(c->d));
    c->d.N = N;
    c->d.M = M;
    c->d.E = (int)E;
    c->d.dc_max = dc_max;
    c->d.divM = fast_div((uint32_t)M);
    c->d.divP = fast_div(1u);
    c->d.divG = fast_div((uint32_t)((N + 3) / 4));
    c->sparse = true;
    c->rate = 1.0 - (double)M / (double)N;
    const size_t words = (size_t)(M + 1) + (size_t)E + (size_t)(N + 1) + (size_t)E;
    if (cudaGetDevice(&c->device) != cudaSuccess || cudaMalloc(&c->sp_mem, words * 4) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        set_error("device allocation of the index tables failed");
        return LDPC_ENOMEM;
    }
    int *dm = (int *)c->sp_mem;
    cudaError_t ce = cudaMemcpy(dm, row_ptr, (size_t)(M + 1) * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(dm + M + 1, col_idx, (size_t)E * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(dm + M + 1 + E, cptr.data(), (size_t)(N + 1) * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(dm + M + 1 + E + N + 1, cedge.data(), (size_t)E * 4, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(c->sp_mem);
        delete c;
        return cuda_fail(ce, "cudaMemcpy(index tables)");
    }
    c->sp.rp = dm;
    c->sp.col = dm + M + 1;
    c->sp.cptr = dm + M + 1 + E;
    c->sp.cedge = dm + M + 1 + E + N + 1;
    c->sp.dc_max = dc_max;
    c->sp.dv_max = dv_max;
    c->h_rp.assign(row_ptr, row_ptr + M + 1);
    c->h_col.assign(col_idx, col_idx + E);
    *out = c;
    return LDPC_OK;
}

ldpc_status ldpc_code_dims(ldpc_code c, int64_t *N, int64_t *M, int64_t *E, int64_t *K) {
    if (!c) {
        set_error("code is NULL");
        return LDPC_EINVAL;
    }
    if (N) *N = c->d.N;
    if (M) *M = c->d.M;
    if (E) *E = c->d.E;
    if (K) *K = (int64_t)c->d.N - c->d.M;
    return LDPC_OK;
}

// the address a kernel uses for p: p itself for device or managed memory, the device mapping of
// pinned (page-locked) host memory, NULL for pageable host memory (or NULL)
static void *mapped_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return const_cast<void *>(p);
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

// Slot count of the streaming decode, or 0 when ldpc_decode keeps its batch path: the stream
// gives every frame exactly the batch path's iterations and decisions (QC codes, sum-product
// with FP32 messages or integer min-sum, early stop -- without it a stream has nothing to
// refill), does not produce posteriors, and pays off once the batch is at least twice the slots.
static int stream_slots(const ldpc_code c, int gamma, const ldpc_decode_opts &o, const float *post) {
    if (c->sparse || !o.early_stop || post) return 0;
    if (!((o.algo == LDPC_ALGO_SP && o.msg == LDPC_MSG_F32) || o.algo == LDPC_ALGO_MS)) return 0;
    const int W = 32 * lanes_per_word(o.msg);
    int slots = c->tuned_slots[o.algo][o.msg];
    if (slots <= 0) slots = 4096;
    slots = (slots + W - 1) / W * W;
    return gamma >= 2 * slots ? slots : 0;
}

ldpc_status ldpc_decode(ldpc_code c, const float *llr, int32_t gamma, const ldpc_decode_opts *opts, float *post,
                        uint8_t *hard, int32_t *iters, int32_t *ok, void *stream) {
    if (!c || !llr || gamma < 1) {
        set_error("need code, llr and gamma >= 1");
        return LDPC_EINVAL;
    }
    ldpc_status st = check_opts(c, opts);
    if (st != LDPC_OK) return st;
    const ldpc_decode_opts &o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    if (const int slots = stream_slots(c, gamma, o, post)) {
        StreamIO io;
        io.llr = (const float *)mapped_ptr(llr);
        io.hard = (uint8_t *)mapped_ptr(hard);
        io.iters = (int32_t *)mapped_ptr(iters);
        io.ok = (int32_t *)mapped_ptr(ok);
        // every buffer device-accessible (device memory or pinned host memory): stream
        if (io.llr && (!hard || io.hard) && (!iters || io.iters) && (!ok || io.ok)) {
            unsigned long long h[8];
            return qc_ber_sim_refill(c, 0.0, 0, 0, gamma, 0, slots, o, h, s, &io);
        }
    }
    const bool host_in = pointer_kind(llr) == 1;
    const bool host_out = (post && pointer_kind(post) == 1) || (hard && pointer_kind(hard) == 1) ||
                          (iters && pointer_kind(iters) == 1) || (ok && pointer_kind(ok) == 1);
    st = qc_ensure_workspace(c, (size_t)gamma, host_in || host_out);
    if (st != LDPC_OK) return st;
    DecodeWs &w = c->ws;
    const size_t NB = (size_t)gamma * c->d.N;
    const float *src = llr;
    if (host_in) {
        LDPC_CUDA_TRY(cudaMemcpyAsync(w.stage_llr, llr, NB * 4, cudaMemcpyHostToDevice, s));
        src = w.stage_llr;
    }
    st = qc_pack_llr(c, src, gamma, o, s);
    if (st != LDPC_OK) return st;
    st = qc_decode_device(c, gamma, o, post != nullptr, s);
    if (st != LDPC_OK) return st;
    float *d_post = post && pointer_kind(post) == 1 ? w.stage_post : post;
    uint8_t *d_hard = hard && pointer_kind(hard) == 1 ? w.stage_hard : hard;
    int32_t *d_iters = iters && pointer_kind(iters) == 1 ? w.stage_i32 : iters;
    int32_t *d_ok = ok && pointer_kind(ok) == 1 ? w.stage_i32 + w.gamma_cap : ok;
    st = qc_unpack_outputs(c, gamma, o, d_post, d_hard, d_iters, d_ok, s);
    if (st != LDPC_OK) return st;
    if (d_post != post) LDPC_CUDA_TRY(cudaMemcpyAsync(post, d_post, NB * 4, cudaMemcpyDeviceToHost, s));
    if (d_hard != hard) LDPC_CUDA_TRY(cudaMemcpyAsync(hard, d_hard, NB, cudaMemcpyDeviceToHost, s));
    if (d_iters != iters) LDPC_CUDA_TRY(cudaMemcpyAsync(iters, d_iters, (size_t)gamma * 4, cudaMemcpyDeviceToHost, s));
    if (d_ok != ok) LDPC_CUDA_TRY(cudaMemcpyAsync(ok, d_ok, (size_t)gamma * 4, cudaMemcpyDeviceToHost, s));
    return LDPC_OK;
}


ldpc_status ldpc_channel(ldpc_code c, double ebn0_db, uint64_t seed, uint64_t first_frame, int32_t gamma,
                         float *llr_out, void *stream) {
    if (!c || !llr_out || gamma < 1 || !std::isfinite(ebn0_db)) {
        set_error("need code, llr_out, gamma >= 1 and a finite Eb/N0");
        return LDPC_EINVAL;
    }
    if (!(c->rate > 0.0)) {
        set_error("design rate K/N = %g is not positive", c->rate);
        return LDPC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool host_out = pointer_kind(llr_out) == 1;
    float *dst = llr_out;
    if (host_out) {
        ldpc_status st = qc_ensure_workspace(c, (size_t)gamma, 1);
        if (st != LDPC_OK) return st;
        dst = c->ws.stage_llr;
    }
    ldpc_status st = qc_channel_frames(c, channel_sigma(c, ebn0_db), seed, first_frame, gamma, dst, s);
    if (st != LDPC_OK) return st;
    if (host_out)
        LDPC_CUDA_TRY(cudaMemcpyAsync(llr_out, dst, (size_t)gamma * c->d.N * 4, cudaMemcpyDeviceToHost, s));
    return LDPC_OK;
}

// candidate slot counts of the autotuner, largest first (the workspace is allocated once)
static const int kTuneSlots[] = {16384, 8192, 4096, 2048, 1024};
constexpr int kTuneCands = 5;

ldpc_status ldpc_tune_slots(ldpc_code c, double ebn0_db, uint64_t seed, const ldpc_decode_opts *opts,
                            int32_t *gamma_out, double *mbit_s, void *stream) {
    if (!c || !gamma_out || !std::isfinite(ebn0_db)) {
        set_error("need code, gamma_out and a finite Eb/N0");
        return LDPC_EINVAL;
    }
    if (c->sparse) {
        set_error("the continuous simulation takes QC codes");
        return LDPC_EUNSUPPORTED;
    }
    ldpc_status st = check_opts(c, opts);
    if (st != LDPC_OK) return st;
    if (!(c->rate > 0.0)) {
        set_error("design rate K/N = %g is not positive", c->rate);
        return LDPC_EINVAL;
    }
    const ldpc_decode_opts &o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    const double sigma = channel_sigma(c, ebn0_db);
    const double K = (double)c->d.N - c->d.M;
    unsigned long long h[8];
    int best = 0;
    double best_rate = -1.0;
    for (int i = 0; i < kTuneCands; ++i) {
        const int slots = kTuneSlots[i];
        // frames of a reserved id range (top bit set): a short run to settle the workspace and
        // caches, then the timed run of four frames per slot
        const uint64_t base = (1ull << 63) + (uint64_t)i * (1ull << 40);
        st = qc_ber_sim_refill(c, sigma, seed, base, slots, 1ll << 60, slots, o, h, s);
        if (st != LDPC_OK) return st;
        const auto t0 = std::chrono::steady_clock::now();
        st = qc_ber_sim_refill(c, sigma, seed, base + (1ull << 39), 4ll * slots, 1ll << 60, slots, o, h, s);
        if (st != LDPC_OK) return st;
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const double rate = sec > 0 ? (double)h[0] * K / sec / 1e6 : 0.0;
        if (mbit_s) mbit_s[i] = rate;
        if (rate > best_rate) best_rate = rate, best = slots;
    }
    c->tuned_slots[o.algo][o.msg] = best;
    *gamma_out = best;
    return LDPC_OK;
}

ldpc_status ldpc_ber_sim(ldpc_code c, double ebn0_db, uint64_t seed, uint64_t first_frame, int64_t max_frames,
                         int64_t target_frame_errors, int32_t gamma, const ldpc_decode_opts *opts,
                         ldpc_ber_result *out, void *stream) {
    if (!c || !out || gamma < 0 || max_frames < 1 || !std::isfinite(ebn0_db)) {
        set_error("need code, out, gamma >= 0, max_frames >= 1 and a finite Eb/N0");
        return LDPC_EINVAL;
    }
    if (gamma == 0 && opts && !c->sparse && opts->algo >= 0 && opts->algo < 3 && opts->msg >= 0 && opts->msg < 3) {
        gamma = c->tuned_slots[opts->algo][opts->msg];
        if (gamma == 0) {
            ldpc_status ts = ldpc_tune_slots(c, ebn0_db, seed, opts, &gamma, nullptr, stream);
            if (ts != LDPC_OK) return ts;
        }
    }
    if (gamma < 1) {
        set_error("gamma must be >= 1, or 0 for the tuned slot count");
        return LDPC_EINVAL;
    }
    if (!(c->rate > 0.0)) {
        set_error("design rate K/N = %g is not positive", c->rate);
        return LDPC_EINVAL;
    }
    if (c->sparse) {
        set_error("ldpc_ber_sim takes QC codes; decode a general code with ldpc_channel + ldpc_decode");
        return LDPC_EUNSUPPORTED;
    }
    ldpc_status st = check_opts(c, opts);
    if (st != LDPC_OK) return st;
    const ldpc_decode_opts &o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    std::memset(out, 0, sizeof(*out));
    const double sigma = channel_sigma(c, ebn0_db);
    unsigned long long h[8];
    // continuous simulation: slots refilled as frames stop
    st = qc_ber_sim_refill(c, sigma, seed, first_frame, max_frames, target_frame_errors, gamma, o, h, s);
    if (st != LDPC_OK) return st;
    out->frames = (int64_t)h[0];
    out->frame_errors = (int64_t)h[1];
    out->bit_errors = (int64_t)h[2];
    out->iters_sum = (int64_t)h[3];
    out->undetected = (int64_t)h[4];
    out->bit_errors_sq = (int64_t)h[5];
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return LDPC_OK;
}

ldpc_status ldpc_phi_eval(const float *x, float *y, int64_t n, int32_t variant, void *stream) {
    if (!x || !y || n < 0 || n > (int64_t)1 << 30 || variant < 0 || variant > 2) {
        set_error("need device x, y, 0 <= n <= 2^30 and variant 0, 1 or 2");
        return LDPC_EINVAL;
    }
    if (pointer_kind(x) != 0 || pointer_kind(y) != 0) {
        set_error("ldpc_phi_eval takes device buffers");
        return LDPC_EINVAL;
    }
    if (n == 0) return LDPC_OK;
    return phi_eval(x, y, (int)n, variant, (cudaStream_t)stream);
}

}  // extern "C"

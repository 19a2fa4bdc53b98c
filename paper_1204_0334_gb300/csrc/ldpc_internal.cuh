// Internal declarations of the sm_103a LDPC library (not part of the C-ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "ldpc.h"

namespace ldpc {

constexpr int kMaxJ = 8;
constexpr int kMaxL = 32;

// Exact n / d for 0 <= n < 2^32 and a divisor d >= 1 fixed for a launch: the multiply-high
// method of Granlund and Montgomery, "Division by invariant integers using multiplication"
// (PLDI 1994, Fig. 4.1): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// t = mulhi(m, n), q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
    uint32_t d, m;
    int s1, s2;
};
inline FastDiv fast_div(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}
// QC code description passed by value to every kernel (lives in the constant
// parameter bank, so warp-uniform reads of shifts and block offsets are broadcasts).
// Block (j, l) with shift a >= 0 owns p edges; edge k of the block joins check
// j*p + ((k - a) mod p) and variable l*p + k ("variable-side" order), so both the
// check pass and the variable pass address edges by arithmetic, not tables.
struct QcDesc {
    int J, L, p;
    int N, M, E;        // variables, checks, edges
    int dc_max;         // largest row degree over the block rows
    int shift[kMaxJ * kMaxL];  // -1 = zero block
    int eoff[kMaxJ * kMaxL];   // first edge of block (j, l), -1 for a zero block
    FastDiv divM, divP, divG;  // n / M, n / p and n / ceil(N / 4) (work-item decomposition)
};

// Device workspace of one code object, grown on demand.  Frames are grouped in
// packages of W = 32 * V frames (V frames per lane, 4 bytes per lane per edge).
struct DecodeWs {
    size_t gamma_cap = 0;      // frames the buffers hold (multiple of 128)
    size_t msg_bytes = 0;
    void *msg = nullptr;       // [P][E][W] edge messages (one kind live at a time)
    void *mu = nullptr;        // [P][N][W] channel LLRs (float, or int8 for MS)
    float *post = nullptr;     // [P][N][W] posteriors (package layout)
    uint32_t *hw = nullptr;    // [P][N][V] hard-decision words, bit = lane
    uint32_t *flags = nullptr; // per package: done[V], unsat[2][V], valid[V], fin[V]
    int32_t *iters = nullptr;  // [gamma_cap] in package order (frame f)
    unsigned long long *counters = nullptr;  // [8] error counters (ber sim)
    int *act = nullptr;        // [1 + P]: count, then the packages with a frame still running
    // host-buffer staging
    float *stage_llr = nullptr;   // [gamma][N]
    float *stage_post = nullptr;  // [gamma][N]
    uint8_t *stage_hard = nullptr;
    int32_t *stage_i32 = nullptr;  // [2][gamma]
};

}  // namespace ldpc

struct ldpc_noms_state;  // training state of the learned min-sum (noms.cu)
struct ldpc_sim_state;   // frame slots of the continuous simulation (sim.cu)
struct ldpc_encoder_s;   // systematic encoder (encode.cu)

namespace ldpc {
// index tables of a general sparse code (device memory): H in compressed-row form with
// edges numbered row by row, and each variable's edges (compressed-column form)
struct SparseTab {
    const int *rp = nullptr;     // [M + 1] first edge of each row
    const int *col = nullptr;    // [E] variable of each edge
    const int *cptr = nullptr;   // [N + 1] first entry of each variable in cedge
    const int *cedge = nullptr;  // [E] edges of each variable, in increasing row order
    int dc_max = 0, dv_max = 0;  // largest row / column degree
};
}  // namespace ldpc

struct ldpc_code_s {
    ldpc::QcDesc d;           // QC description; for a sparse code only N, M, E are set (J = 0)
    bool sparse = false;
    ldpc::SparseTab sp;       // sparse code: the index tables
    void *sp_mem = nullptr;   // their device allocation
    ldpc_noms_state *noms = nullptr;
    ldpc_sim_state *sim = nullptr;
    ldpc_encoder_s *enc = nullptr;   // built on first use, under enc_mu
    std::mutex enc_mu;
    std::vector<int> h_rp, h_col;    // sparse code: H in compressed-row form (host copy)
    int device = 0;
    double rate = 0.0;   // design rate K/N
    int tuned_slots[3][3] = {};      // slot count picked by ldpc_tune_slots, per [algo][msg] (0 = not tuned)
    ldpc::DecodeWs ws;
};

namespace ldpc {

// thread-local error text
void set_error(const char *fmt, ...);
ldpc_status cuda_fail(cudaError_t e, const char *what);

#define LDPC_CUDA_TRY(call)                                   \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return ::ldpc::cuda_fail(_e, #call); \
    } while (0)

// 0: device pointer (or managed); 1: host pointer; -1: null
int pointer_kind(const void *p);
// validation of decode options shared by every decode entry point (LDPC_OK or the error)
ldpc_status check_opts(const ldpc_code c, const ldpc_decode_opts *o);
// noise level of Eb/N0 (dB) at the code's design rate: sigma^2 = 1 / (2 R 10^(EbN0/10))
double channel_sigma(const ldpc_code c, double ebn0_db);

// sizes of the flags block per package
inline int flags_per_package(int V) { return 5 * V; }

// launchers implemented in qc_decode.cu
ldpc_status qc_ensure_workspace(ldpc_code c, size_t gamma, int want_host_stage);
ldpc_status qc_decode_device(ldpc_code c, int gamma, const ldpc_decode_opts &o, bool want_post,
                             cudaStream_t s);
ldpc_status qc_pack_llr(ldpc_code c, const float *llr, int gamma, const ldpc_decode_opts &o, cudaStream_t s);
ldpc_status qc_unpack_outputs(ldpc_code c, int gamma, const ldpc_decode_opts &o, float *post, uint8_t *hard,
                              int32_t *iters, int32_t *ok, cudaStream_t s);
ldpc_status qc_channel_frames(ldpc_code c, double sigma, uint64_t seed, uint64_t first_frame, int gamma,
                              float *out, cudaStream_t s);
// syndrome of the hard decisions into flag word `word` (+v) of every package
ldpc_status qc_syndrome(ldpc_code c, int P, int V, int word, cudaStream_t s);

ldpc_status phi_eval(const float *x, float *y, int n, int variant, cudaStream_t s);
void noms_free(ldpc_noms_state *w);
// pipelined node passes (qc_pipe.cu)
// fresh (continuous simulation, else NULL): per package [2V] words, bits V..2V-1 mark
// frames that entered their slot this step; their outgoing messages are set to 0
// ages (continuous simulation, learned min-sum): per slot, the iteration each frame runs in
// this pass (1-based); its parameter row is ages - 1, clamped to [0, max_iter)
ldpc_status qc_cn_pipe(ldpc_code c, const ldpc_decode_opts &o, int it, cudaStream_t s,
                       const uint32_t *fresh = nullptr, const int *ages = nullptr);
ldpc_status qc_vn_pipe(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                       cudaStream_t s);
// packages with a running frame
ldpc_status qc_compact(ldpc_code c, int P, int V, cudaStream_t s);
// general (index-table) codes (qc_pipe.cu, sparse.cu)
ldpc_status qc_cn_pipe_sparse(ldpc_code c, const ldpc_decode_opts &o, cudaStream_t s);
ldpc_status qc_vn_pipe_sparse(ldpc_code c, const ldpc_decode_opts &o, bool stop, bool post, int it, int par,
                              cudaStream_t s);
ldpc_status sparse_decode_device(ldpc_code c, int gamma, const ldpc_decode_opts &o, bool want_post, cudaStream_t s);
ldpc_status qc_init_flags(ldpc_code c, int gamma, int V, cudaStream_t s);
ldpc_status qc_finish_frames(ldpc_code c, int gamma, const ldpc_decode_opts &o, cudaStream_t s);
// continuous simulation (sim.cu)
void sim_free(ldpc_sim_state *st);
// streaming decode (ldpc_decode): the caller's [gamma][N] channel LLRs (device-accessible) and
// the outputs each frame writes as it retires (NULL = not wanted)
struct StreamIO {
    const float *llr;
    uint8_t *hard;
    int32_t *iters, *ok;
};
ldpc_status qc_ber_sim_refill(ldpc_code c, double sigma, uint64_t seed, uint64_t first_frame, int64_t max_frames,
                              int64_t target, int gamma, const ldpc_decode_opts &o, unsigned long long *h,
                              cudaStream_t s, const StreamIO *io = nullptr);

// systematic encoder (encode.cu)
void enc_free(ldpc_encoder_s *e);
// host part (information set, parity matrix); no device memory
ldpc_status enc_build_host(ldpc_code c);
// device tables and a sliced-codeword scratch for `groups` groups of 32 frames
ldpc_status enc_ensure_device(ldpc_code c, size_t groups);
int64_t enc_k(const ldpc_code c);
int enc_words(const ldpc_code c);  // ceil(N / 32): words of a frame-major codeword row
// continuous simulation with random codewords: wrong information bits of the frames that
// retire this step (from the staged decisions, before a new frame's overwrite them), and
// the codewords of the frames that enter a slot (frame-major rows cwf[slot][enc_words])
ldpc_status enc_sim_errors(ldpc_code c, int P, int V, const uint32_t *sflags, const uint32_t *cwf, int *errs,
                           cudaStream_t s);
ldpc_status enc_sim_codewords(ldpc_code c, int slots, const int *rlist, const int *rcount, int parity,
                              const uint64_t *fid, uint64_t seed, uint32_t *cwf, cudaStream_t s);

inline int lanes_per_word(int msg) { return msg == LDPC_MSG_F32 ? 1 : (msg == LDPC_MSG_F16 ? 2 : 4); }

}  // namespace ldpc

namespace ldpc {
// launch accounting and optional per-launch event timing (profile.cu)
void count_launch(int n = 1);
bool profiling();
// kind 0 = check node, 1 = variable node; returns a slot for prof_end (or -1)
int prof_begin(int kind, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);
}  // namespace ldpc

/*
 * ldpc.h -- C-ABI of the GB300 (sm_103a) batched belief-propagation decoders
 * for quasi-cyclic LDPC block codes and the LDPC convolutional codes derived
 * from them (Zhao & Lau, arXiv 1204.0334).
 *
 * Conventions for every call:
 *  - Plain C types only.  Buffers are caller-owned.  Unless a parameter says
 *    otherwise, a buffer may live in device memory or in host memory (pinned
 *    or pageable); the library finds out with cudaPointerGetAttributes and
 *    stages host buffers through its own device workspace.  Results written
 *    to host buffers are valid once `stream` has been synchronized.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is enqueued on it; calls return without
 *    waiting unless stated.
 *  - Objects (ldpc_code, ldpccc) are owned by the library, created on the
 *    current CUDA device and used on that device only.  One object must not
 *    be used from two streams or threads at the same time: it owns the
 *    workspace its calls use.
 *  - Every call returns an ldpc_status; no exception crosses the ABI.  On an
 *    error, ldpc_last_error() gives a thread-local description.
 *  - Frames are laid out frame-major: element (f, n) of an [gamma][N] buffer
 *    is at f*N + n.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDPC_OK = 0,
    LDPC_EINVAL = 1,        /* bad argument: sizes, null pointers, shifts out of range */
    LDPC_ENOMEM = 2,        /* device or host allocation failed */
    LDPC_ECUDA = 3,         /* a CUDA runtime call failed (detail in ldpc_last_error) */
    LDPC_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
    LDPC_EUNSUPPORTED = 5   /* valid request this build does not implement */
} ldpc_status;

typedef struct ldpc_code_s *ldpc_code;
typedef struct ldpccc_s *ldpccc;
typedef struct ldpc_batch_s *ldpc_batch;

/* Check-node rule. */
enum {
    LDPC_ALGO_SP = 0,   /* sum-product, eq. (bphs) of Algorithm 1, log-domain phi form in FP32 */
    LDPC_ALGO_MS = 1,   /* integer min-sum over int8 messages (quantized LLRs, F fractional bits) */
    LDPC_ALGO_NOMS = 2  /* normalized/offset min-sum with per-iteration, per-circulant (w, o) */
};

/* Storage type of the edge messages (arithmetic is FP32 for SP/NOMS, int32 for MS). */
enum { LDPC_MSG_F32 = 0, LDPC_MSG_F16 = 1, LDPC_MSG_I8 = 2 };

typedef struct {
    int32_t max_iter;          /* I_max >= 1: iterations of Algorithm 1 */
    int32_t early_stop;        /* 1: a frame stops at the first iteration i >= 1 whose hard
                                  decisions satisfy every check; its outputs are those of i */
    int32_t algo;              /* LDPC_ALGO_* */
    int32_t msg;               /* LDPC_MSG_*; MS requires LDPC_MSG_I8, SP/NOMS take F32 or F16 */
    float clip;                /* SP/NOMS: channel LLRs, messages and posteriors are clipped to
                                  [-clip, clip] (default 30) */
    int32_t frac_bits;         /* MS: q = clamp(rint(mu * 2^frac_bits), -127, 127) (default 2) */
    const float *noms_params;  /* NOMS: device [max_iter][J*L][2] of (w, o), 8-byte aligned
                                  (LDPC_EINVAL otherwise); else NULL */
    int32_t codewords;         /* ldpc_ber_sim only: LDPC_CODEWORDS_ZERO (default) or
                                  LDPC_CODEWORDS_RANDOM; the other calls ignore it */
    int32_t reserved[3];       /* must be zero */
} ldpc_decode_opts;

/* Transmitted codewords of ldpc_ber_sim. */
enum { LDPC_CODEWORDS_ZERO = 0, LDPC_CODEWORDS_RANDOM = 1 };

/* Defaults: max_iter 30, early_stop 0, SP, F32 messages, clip 30, frac_bits 2. */
void ldpc_default_opts(ldpc_decode_opts *opts);

const char *ldpc_status_str(ldpc_status s);
/* Thread-local text of the last error raised in this thread ("" if none). */
const char *ldpc_last_error(void);

/*
 * ldpc_code_create -- a (J, L) QC-LDPC code, eq. (qcH) of Sec. II-A.
 *   shifts: host int32 [J][L] row-major; a_jl in [0, p) selects the circulant
 *           whose row r has its one in column (r + a_jl) mod p (the identity
 *           shifted right a_jl times); -1 selects the zero block (the "shift
 *           number" convention of Sec. IV-B-1).  Copied; the caller keeps it.
 *   J, L:   1 <= J <= 8, 1 <= L <= 32; p >= 1; J*L*p*... must fit in int32.
 *   N = L p variables, M = J p checks, E = p * (number of non-zero blocks).
 * Uses the current CUDA device.  Errors: LDPC_EINVAL (sizes, shift range,
 * out == NULL), LDPC_ENOMEM.
 */
ldpc_status ldpc_code_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, ldpc_code *out);
/*
 * ldpc_code_create_sparse -- a general (not quasi-cyclic) LDPC code given by its
 * parity-check matrix H (Sec. II-A), for decoders that gather through index tables as
 * the paper's LUT_c / LUT_v do (Sec. IV-A) instead of circulant address arithmetic.
 *   row_ptr: host int32 [M + 1], col_idx: host int32 [E] -- H in compressed-row form:
 *            the ones of check m sit in columns col_idx[row_ptr[m] .. row_ptr[m+1]),
 *            strictly increasing within a row; edges are numbered row by row (the
 *            paper's order, eq. simpleH).  Copied; the caller keeps them.
 *   Limits: 1 <= M, N; every row degree in [1, 32]; every column degree in [0, 8];
 *   E * 32 < 2^31.
 * ldpc_decode, ldpc_decode_noalloc and ldpc_channel accept the code; ldpc_ber_sim,
 * the learned min-sum, heterogeneous batches and LDPCCC derivation take QC codes only
 * (LDPC_EUNSUPPORTED).  Errors: LDPC_EINVAL (sizes, indices, degrees), LDPC_ENOMEM.
 */
ldpc_status ldpc_code_create_sparse(int32_t M, int32_t N, const int32_t *row_ptr, const int32_t *col_idx,
                                    ldpc_code *out);
ldpc_status ldpc_code_destroy(ldpc_code code);
/* N, M, E and the design information length K = N - M (any pointer may be NULL). */
ldpc_status ldpc_code_dims(ldpc_code code, int64_t *N, int64_t *M, int64_t *E, int64_t *K);

/*
 * ldpc_decode -- Algorithm 1 (Sec. II-B) on gamma frames at once (the
 * paper's Gamma-codeword batches, Sec. IV-A).
 *   llr:   [gamma][N] float channel LLRs mu_n = ln P(c_n=0|y_n)/P(c_n=1|y_n).
 *   post:  [gamma][N] float a-posteriori LLRs beta_n of eq. (bpd), or NULL.
 *          SP/NOMS: clipped to +-clip.  MS: the integer posterior q + sum(alpha)
 *          times 2^-frac_bits.
 *   hard:  [gamma][N] uint8 hard decisions of eq. (hrddcs) (1 iff beta_n < 0), or NULL.
 *   iters: [gamma] int32 iterations run per frame, or NULL.
 *   ok:    [gamma] int32, 1 iff the hard decisions satisfy every check, or NULL.
 * gamma >= 1 (any value; internally padded to the package width).
 * Streaming: for a QC code with opts->early_stop, sum-product with F32 messages
 * or integer min-sum, post == NULL, gamma at least twice the slot count (the
 * one ldpc_tune_slots picked for this code and algo/msg, else 4096) and every
 * buffer in device or pinned host memory, the frames stream through that many
 * slots as in ldpc_ber_sim: a frame enters a slot as soon as the previous one
 * stops, reading its LLR row directly (pinned host rows through their device
 * mapping, no staging copy), and writes its decisions, iteration count and ok
 * flag when it stops.  Each frame gets exactly the iterations and decisions of
 * the batch path.  This form returns when the batch is decoded (it synchronizes
 * the stream).
 * Errors: LDPC_EINVAL (null code/llr, gamma < 1, bad opts), LDPC_EUNSUPPORTED
 * (algo/msg pair not built), LDPC_ENOMEM, LDPC_ECUDA, LDPC_ETIMEOUT.
 */
ldpc_status ldpc_decode(ldpc_code code, const float *llr, int32_t gamma, const ldpc_decode_opts *opts,
                        float *post, uint8_t *hard, int32_t *iters, int32_t *ok, void *stream);

/*
 * ldpc_decode_noalloc -- ldpc_decode for callers that cannot allocate device
 * memory (for example code running under a stream capture that must not add
 * allocation nodes, real-time loops that cannot afford a synchronous
 * cudaMalloc, or processes whose device memory is reserved up front by another
 * allocator).  The paper has no counterpart.  Same arguments and results as
 * ldpc_decode, but every buffer must be device memory and the decoder's
 * workspace comes from a fixed 16 MiB array inside the library (held on every
 * GPU that loads it until the process exits); the call itself calls no
 * cudaMalloc/cudaFree.  A decode of gamma frames needs about
 * (4E + 8N + N/8) * gamma bytes (rounded up to 128 frames): requests beyond
 * the array return LDPC_EINVAL with the size in ldpc_last_error().  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the array, and each decode initializes what it reads, but
 * calls whose GPU work overlaps (other streams or threads) race on it.
 * Sum-product (F32/F16 storage) and integer min-sum; LDPC_EUNSUPPORTED for NOMS.
 */
ldpc_status ldpc_decode_noalloc(ldpc_code code, const float *llr, int32_t gamma, const ldpc_decode_opts *opts,
                                float *post, uint8_t *hard, int32_t *iters, int32_t *ok, void *stream);

/*
 * Heterogeneous batches (no paper counterpart; the paper decodes one code at a
 * time, Sec. IV-A).  ldpc_batch_create plans a batch of ncodes QC codes (J <= 4,
 * L <= 24), code i with gammas[i] frames, all decoded with the same options
 * (sum-product with F32/F16 storage or integer min-sum; early stop as in
 * opts).  The codes must outlive the batch.  The batch owns one device
 * workspace for all codes.  ldpc_batch_decode runs Algorithm 1 on every code
 * with a shared iteration loop: per iteration one check-pass and one
 * variable-pass launch over the tiles (code, package, row/variable range) of
 * every package that still has a running frame, listed again after each
 * variable pass.  With early stop, after iteration K the frames of a code that
 * are still running, when they are at most three quarters of its frames, move
 * densely into a second package area of that code (frame-level compaction), so
 * later iterations visit only their packages; their outputs are written back
 * to their own rows.  The workspace holds both areas.  The loop is captured
 * into a CUDA graph on the second call and replayed afterwards; the first call
 * also tunes the tile sizes by timing three candidates on its frames
 * (ldpc_batch_info reports the choice) and, unless set, K among none, 8, 12
 * and 16 by timing whole decodes (ldpc_batch_compaction).  With compaction in
 * use a call first waits until the previous call on the batch has copied its
 * output pointer arrays.
 *   llr: host array of ncodes device pointers, [gammas[i]][N_i] float each.
 *   hard / iters / ok: host arrays of ncodes device pointers (entries or the
 *   arrays may be NULL): [gammas[i]][N_i] uint8, [gammas[i]] int32, int32.
 * Errors: LDPC_EINVAL, LDPC_EUNSUPPORTED (NOMS, larger degrees), LDPC_ENOMEM.
 */
ldpc_status ldpc_batch_create(const ldpc_code *codes, int32_t ncodes, const int32_t *gammas,
                              const ldpc_decode_opts *opts, ldpc_batch *out);
ldpc_status ldpc_batch_decode(ldpc_batch batch, const float *const *llr, uint8_t *const *hard,
                              int32_t *const *iters, int32_t *const *ok, void *stream);
/* tile rows of the check pass, variable groups of the variable pass, tuning times (ms) of the 3 candidates */
ldpc_status ldpc_batch_info(ldpc_batch batch, int32_t *tile_rows, int32_t *tile_groups, double *tune_ms3);
/* frames of each code the last ldpc_batch_decode moved to its second area (host int32[ncodes]; 0 for
   codes left in place); synchronizes the stream of that decode */
ldpc_status ldpc_batch_moved(ldpc_batch batch, int32_t *moved);
/* the compaction point: after_iter >= 1 compacts after that iteration, 0 never, -1 lets the next
   decode's autotuner choose (the default); resets the captured graph.  Errors: LDPC_EINVAL. */
ldpc_status ldpc_batch_set_compaction(ldpc_batch batch, int32_t after_iter);
/* the compaction point in use and the autotuner's whole-decode times (ms) for none, 8, 12, 16
   (host double[4] or NULL; 0 where a candidate was not timed) */
ldpc_status ldpc_batch_compaction(ldpc_batch batch, int32_t *after_iter, double *tune_ms4);
ldpc_status ldpc_batch_destroy(ldpc_batch batch);

/*
 * ldpc_channel -- the device-side channel of Sec. V (codeword and noise made
 * on the GPU): the all-zero codeword sent as BPSK x = +1 over AWGN, Sec. II-B,
 * y = 1 + sigma g, mu = 2 y / sigma^2, with sigma^2 = 1 / (2 R 10^(EbN0/10))
 * and R = K/N the design rate.  g is Box-Muller on Philox4x32-10 words:
 * bit n of frame F uses counter (n/4, F mod 2^32, F / 2^32, 0) under key
 * (seed mod 2^32, seed / 2^32); word w -> u = (floor(w / 2^9) + 1/2) 2^-23;
 * words (0,1) and (2,3) give the normals of bits 4q, 4q+1 and 4q+2, 4q+3 as
 * (r cos 2 pi u', r sin 2 pi u'), r = sqrt(-2 ln u).
 *   llr_out: [gamma][N] float, frames first_frame .. first_frame+gamma-1.
 */
ldpc_status ldpc_channel(ldpc_code code, double ebn0_db, uint64_t seed, uint64_t first_frame, int32_t gamma,
                         float *llr_out, void *stream);

/*
 * Systematic encoding: the transmitted codewords of Sec. V, made on the device.
 *
 * Information set.  Scanning the columns of H from n = N-1 down to 0, column n
 * is a parity position when it is not in the GF(2) span of the columns to its
 * right, else an information position.  The parity columns are a basis of
 * H's column space, so k = N - rank(H) >= K = N - M, and for every u in
 * {0,1}^k exactly one codeword c (H c = 0) has c[info_pos[j]] = u[j], with
 * info_pos increasing.  The encoder is built on the host by Gauss-Jordan
 * elimination over GF(2) the first time a call below needs it (O(M^2 N / 64)
 * word operations: about a second for n = 18360); each frame's parity bits are
 * then a dense GF(2) matrix-vector product on the device.
 *
 * ldpc_code_info_set -- k and, when info_pos != NULL, the k information
 *   positions (host int32 [k]).  Host-only work; no device memory is touched.
 * ldpc_encode -- cw[f] = the codeword of info[f] (device uint8 [gamma][k]; bit
 *   = byte & 1) into device uint8 [gamma][N] (0/1).  info may be NULL when k = 0.
 * ldpc_random_codewords -- the codewords ldpc_ber_sim sends with
 *   LDPC_CODEWORDS_RANDOM: information bit j of frame F is bit j mod 32 of word
 *   (j/32) mod 4 of Philox4x32-10 at counter (j/128, F mod 2^32, F / 2^32, 1)
 *   under key (seed mod 2^32, seed / 2^32) (the channel's counters carry 0 in
 *   the last word); frames first_frame .. first_frame+gamma-1.  info (device
 *   uint8 [gamma][k]) may be NULL; cw as in ldpc_encode.
 * ldpc_channel_codewords -- ldpc_channel with the codeword cw (device uint8
 *   [gamma][N], 0/1) sent as BPSK x = 1 - 2c: mu = 2 (x + sigma g) / sigma^2
 *   with the same g, so an all-zero cw reproduces ldpc_channel exactly.
 * All pointers but info_pos are device pointers (host pointers: LDPC_EINVAL).
 */
ldpc_status ldpc_code_info_set(ldpc_code code, int64_t *k, int32_t *info_pos);
ldpc_status ldpc_encode(ldpc_code code, const uint8_t *info, int32_t gamma, uint8_t *cw, void *stream);
ldpc_status ldpc_random_codewords(ldpc_code code, uint64_t seed, uint64_t first_frame, int32_t gamma,
                                  uint8_t *info, uint8_t *cw, void *stream);
ldpc_status ldpc_channel_codewords(ldpc_code code, double ebn0_db, uint64_t seed, uint64_t first_frame,
                                   int32_t gamma, const uint8_t *cw, float *llr_out, void *stream);

typedef struct {
    int64_t frames;        /* frames decoded */
    int64_t frame_errors;  /* frames with >= 1 wrong bit (all N coded bits counted; with
                              LDPC_CODEWORDS_RANDOM the k information bits) */
    int64_t bit_errors;    /* wrong coded bits (LDPC_CODEWORDS_RANDOM: wrong information bits) */
    int64_t iters_sum;     /* sum over frames of the iterations run */
    int64_t undetected;    /* frames with ok = 1 but >= 1 wrong bit */
    double seconds;        /* wall time of the call */
    int64_t bit_errors_sq; /* sum over frames of (the frame's wrong bits)^2: with bit_errors,
                              the frame-level variance behind a confidence interval of the
                              BER (the bits of one frame do not fail independently) */
} ldpc_ber_result;

/*
 * ldpc_ber_sim -- the Monte-Carlo protocol of Sec. V: fixed iteration cap,
 * frames generated and decoded on the device, error counts reduced on the
 * device.  The decoders run continuously: gamma frame slots (rounded up to
 * whole packages of 32 V frames), and a slot takes the next frame in the
 * step after its frame stops (when opts->early_stop, its decisions satisfy
 * every check, tested after each complete iteration i >= 1; or the iteration
 * cap), so each frame gets exactly the
 * iterations and decisions that ldpc_decode gives it (learned NOMS: each
 * frame's iteration i uses parameter row i).
 * Once frame_errors >= target_frame_errors (the paper uses 100) no new frame
 * starts and the frames in flight finish; at most max_frames frames start.
 * The frames counted are always first_frame .. first_frame + out->frames - 1,
 * drawn exactly as ldpc_channel draws them (opts->codewords =
 * LDPC_CODEWORDS_RANDOM: as ldpc_random_codewords and ldpc_channel_codewords
 * draw them, errors counted over the information bits), so a run can be
 * resumed from (seed, first_frame + out->frames) and partial results added.
 * Blocks the calling thread until the run ends (it reads the totals every
 * two steps).
 *   gamma: frame slots; 0 = the slot count ldpc_tune_slots picked for this code and
 *   opts->algo / opts->msg (tuned on the spot, at this Eb/N0 and seed, if it has not been).
 *   out: host pointer, filled on return.
 */
ldpc_status ldpc_ber_sim(ldpc_code code, double ebn0_db, uint64_t seed, uint64_t first_frame, int64_t max_frames,
                         int64_t target_frame_errors, int32_t gamma, const ldpc_decode_opts *opts,
                         ldpc_ber_result *out, void *stream);
/*
 * ldpc_tune_slots -- the autotuner of the continuous simulation's slot count Gamma
 * (no paper counterpart; the paper fixes Gamma = 32 for its GPU, Sec. IV-A).  Times
 * ldpc_ber_sim's decoding at 16384, 8192, 4096, 2048 and 1024 slots (a settling run
 * of one frame per slot, then a timed run of four frames per slot, frames drawn from
 * the reserved id range [2^63, 2^63 + 2^43), which the caller's runs should avoid) and
 * keeps the fastest in the code object for opts->algo / opts->msg.
 *   gamma_out: host int32, the slot count picked; mbit_s: host double[5] (decoded
 *   information Mbit/s of each candidate, in the order above) or NULL.
 * Synchronizes the stream; grows the code's workspace to 16384 slots.
 * Errors: as ldpc_ber_sim.
 */
ldpc_status ldpc_tune_slots(ldpc_code code, double ebn0_db, uint64_t seed, const ldpc_decode_opts *opts,
                            int32_t *gamma_out, double *mbit_s, void *stream);

/*
 * LDPC convolutional codes derived from a QC base (Sec. II-D): partition H_QC
 * into Lambda x Lambda sub-blocks, Lambda = gcd(J, L), keep the lower part H^L
 * and paste the strictly-upper part H^U below it, repeat down the diagonal.
 * Frames carry c = (L/Lambda) p bits, check layers (J/Lambda) p checks, rate
 * b/c with b = ((L-J)/Lambda) p, syndrome-former memory ms = Lambda - 1.
 *
 * ldpccc_create -- a pipelined decoder (Algorithm 2, Sec. II-E) with I
 *   processors (one per iteration) for gamma independent code streams.  The
 *   shifts follow ldpc_code_create (copied).  Device memory: a ring of
 *   I*Lambda frames holding the channel LLRs and the J*c edge messages of each
 *   frame for all streams (Sec. IV-B-1: I*E message units, E = J L p).
 *   Lambda = 1 (gcd(J, L) = 1) is accepted: frames then decode independently
 *   with I iterations.  Errors: LDPC_EINVAL, LDPC_ENOMEM.
 */
ldpc_status ldpccc_create(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                          ldpccc *out);
/*
 * ldpccc_create_tanner -- the same pipelined decoder for the time-invariant
 * LDPCCC whose polynomial parity-check matrix is [D^{a_jl}] (the unwrapping of
 * a QC base with its shifts as delays, Tanner et al. 2004, which Sec. II-D
 * cites as another construction without specifying it): check j
 * at time instant t involves bit l at instant t - a_jl (a_jl = -1: none), so
 * the syndrome-former memory in instants is the largest shift.  Frames are p
 * instants (c = L p bits, layers of J p checks, b = (L - J) p), which makes the
 * code a memory-1 LDPCCC (ms = 1; 0 when every shift is 0) with one frame type
 * (ldpccc_dims reports Lambda = 1); every other call behaves as for
 * ldpccc_create, with Lambda read as ms + 1 in the slot arithmetic.
 */
ldpc_status ldpccc_create_tanner(const int32_t *shifts, int32_t J, int32_t L, int32_t p, int32_t I, int32_t gamma,
                                 ldpccc *out);
ldpc_status ldpccc_destroy(ldpccc cc);
/* c, b, ms and Lambda (the period in frames) of the code (any pointer may be NULL). */
ldpc_status ldpccc_dims(ldpccc cc, int32_t *c, int32_t *b, int32_t *ms, int32_t *lambda);
/* Empty the pipeline: the next window's first frame is frame 0 of every stream. */
ldpc_status ldpccc_reset(ldpccc cc);
/*
 * ldpccc_decode_window -- T time slots of Algorithm 2: at each slot the next
 * frame of every stream enters processor 1, the I check layers and then the I
 * frames in the decoder are updated (eqs. ldpccc_bph, ldpccc_bpvs), and the
 * frame leaving processor I is decided (eq. ldpccc_hrddcs).  Frame f is decided
 * at slot f + I*(ms+1) - 1, so the first I*(ms+1) - 1 slots after a reset emit
 * nothing; the decoder state carries over to the next call (continuous decoding).
 *   llr:   [gamma][T][c] float channel LLRs of the T arriving frames (mu = 2y/sigma^2).
 *   clip:  LLR clip (e.g. 30), applied to channel LLRs, messages and posteriors.
 *   hard:  [gamma][T][c] uint8 or NULL: the decided frames, stream-major, frame q at [s][q][.].
 *   post:  [gamma][T][c] float or NULL: their a-posteriori LLRs.
 *   first_out: index of the first decided frame (or -1); n_out: number decided (host ints).
 */
ldpc_status ldpccc_decode_window(ldpccc cc, const float *llr, int32_t T, float clip, uint8_t *hard, float *post,
                                 int64_t *first_out, int32_t *n_out, void *stream);

/*
 * ldpccc_channel -- channel LLRs for frames first_frame .. first_frame+T-1 of
 * every stream: all-zero frames over BPSK/AWGN (Sec. II-E: x = 1 - 2v, y = x + g,
 * sigma^2 = 1 / (2 (b/c) 10^(EbN0/10))), mu = 2y/sigma^2.  Bit n of frame f of
 * stream s uses Philox4x32-10 counter (n/4, f mod 2^32, s, 1) under key
 * (seed mod 2^32, seed / 2^32), then Box-Muller as in ldpc_channel.
 *   llr_out: device [gamma][T][c] float.
 */
ldpc_status ldpccc_channel(ldpccc cc, double ebn0_db, uint64_t seed, int64_t first_frame, int32_t T,
                           float *llr_out, void *stream);

/*
 * Learned normalized/offset min-sum (NOMS).  The paper cites reduced-complexity
 * BP (Sec. II-B) without defining it; this is the parameterized min-sum
 *   alpha_e = sign * min(max(w_{l,c(e)} * m_e - o_{l,c(e)}, 0), clip),  m_e = min_{e' != e} |beta_e'|
 * (every message is clipped at +-clip, as in the other decoders: the clip on alpha
 * acts only where w * m_e - o > clip, e.g. for w > 1 and saturated inputs)
 * with one (w, o) per iteration l and circulant block c = j*L + l, used with
 * the variable rule of eq. (bpvs) (clipped at +-clip) for T iterations.
 * Inference: ldpc_decode / ldpc_ber_sim with opts.algo = LDPC_ALGO_NOMS and
 * opts.noms_params = device [max_iter][J*L][2].
 *
 * ldpc_noms_forward -- training forward pass over B frames:
 *   loss = 1/(T N B) sum over iterations l, bits n, frames of softplus(-post^(l)_n)
 *   (BCE of every iteration's posterior against the all-zero codeword).
 *   llr: device [B][N] float; params: device [T][J*L][2] float (w, o), 8-byte aligned
 *   (LDPC_EINVAL otherwise); msg: LDPC_MSG_F32
 *   or LDPC_MSG_F16 storage of the saved messages; ckpt_every = k: the messages of every
 *   k-th iteration are kept and the others recomputed in the backward pass (the
 *   posteriors of every iteration, 4 N bytes per frame, and one bit per edge and frame
 *   are kept as well, so check messages are never recomputed);
 *   loss: device float[1]; post: device [B][N] float (post^(T)) or NULL.
 *   The code object keeps the state for the following ldpc_noms_backward.
 * ldpc_noms_backward -- d loss / d params accumulated into grad (device [T][J*L][2],
 *   the caller zeroes it).  Needs the forward of the same params on the same code
 *   object just before.  Reverse mode written out by hand: through the arg-min edge
 *   of each m_e (lowest index among ties), through min(max(., 0), clip) where that is
 *   positive and below clip, and through the clip of beta where inactive.
 * Errors: LDPC_EINVAL (sizes, host pointers, backward without forward), LDPC_ENOMEM.
 */
ldpc_status ldpc_noms_forward(ldpc_code code, const float *llr, int32_t B, int32_t T, const float *params,
                              int32_t msg, int32_t ckpt_every, float clip, float *loss, float *post, void *stream);
ldpc_status ldpc_noms_backward(ldpc_code code, const float *params, float *grad, void *stream);

/*
 * ldpc_phi_eval -- the check-node transform of the sum-product rule on its own:
 * phi(x) = -ln tanh(x/2) for x >= 0, with which eq. (bphs) reads
 * alpha = prod(sign) * phi(sum_{n' != n} phi(|beta_n'|)) (phi is its own inverse).
 * Exposed so that its accuracy can be checked against the definition.
 *   x, y: device float [n]; variant 0 = the decoder's SFU-based evaluation,
 *   variant 1 = CUDA's expm1f/log1pf form, variant 2 = the decoder's evaluation
 *   on packed pairs (consecutive elements; bit-identical to variant 0 by
 *   construction).  Errors: LDPC_EINVAL.
 */
ldpc_status ldpc_phi_eval(const float *x, float *y, int64_t n, int32_t variant, void *stream);

/*
 * Measurement aid (the paper has no counterpart; its timings are wall-clock
 * totals, Sec. V).  While enabled, each check-node and variable-node kernel
 * launch of the block-code decoder is bracketed by CUDA events on its own
 * stream.  ldpc_profile_read synchronizes those events and returns the summed
 * device time per kind.  `launches` counts every kernel this library has
 * launched since the last ldpc_profile_enable call, enabled or not.
 * Not thread-safe; enable/read from the thread that issues the decodes.
 */
typedef struct {
    int64_t launches;     /* all kernels launched by the library */
    int64_t cn_launches;  /* timed check-node launches */
    double cn_ms;         /* their summed device time */
    int64_t vn_launches;  /* timed variable-node launches */
    double vn_ms;
} ldpc_profile;

ldpc_status ldpc_profile_enable(int32_t on);  /* resets all counters */
ldpc_status ldpc_profile_read(ldpc_profile *out);

/*
 * ldpc_bandwidth_probe -- measurement aid (no paper counterpart): the memory
 * bandwidth a plain streaming kernel of this library reaches, as the peak that
 * the decoders' L2 byte rates are compared with.  mode 0 reads `bytes` of src
 * `reps` times through L2 (ld.global.cg, all sweeps in one launch; a buffer
 * smaller than L2 is then served by L2) and writes one word per thread block to
 * dst (at least 4 * 8 * SM-count bytes); mode 1 copies src to dst `reps` times
 * (one launch each, read + write bytes counted).  One untimed sweep precedes
 * the timed ones; the time comes from CUDA events on `stream`, and
 * *gbs_out = bytes moved / time / 1e9.
 * src, dst: device buffers, 16-byte aligned; bytes a positive multiple of 16;
 * bytes * reps below 2^38.
 * Synchronizes the stream.  Errors: LDPC_EINVAL, LDPC_ECUDA.
 */
ldpc_status ldpc_bandwidth_probe(const void *src, void *dst, int64_t bytes, int32_t reps, int32_t mode,
                                 double *gbs_out, void *stream);

/*
 * ldpc_sync_probe -- measurement aid (no paper counterpart): what one phase
 * boundary of an iteration loop of persistent passes costs, done two ways with
 * no work in the phases.  (a) `boundaries` back-to-back launches of an empty
 * kernel (grids of 1, 4, 2 and 3 blocks per SM in turn, as the heterogeneous
 * batch's tile, syndrome, check and variable passes), captured once in a CUDA
 * graph and replayed `reps` times; (b) one cooperative kernel (two resident
 * blocks of 256 threads per SM) with `boundaries` grid-wide barriers, launched
 * `reps` times.  *graph_us and *coop_us: microseconds per boundary (CUDA events
 * on a private stream, after three untimed runs of each).
 * 1 <= boundaries <= 4096, 1 <= reps <= 10000.  Synchronizes the device's work on
 * its own stream only.  Errors: LDPC_EINVAL, LDPC_EUNSUPPORTED (no cooperative
 * launch), LDPC_ECUDA.
 */
ldpc_status ldpc_sync_probe(int32_t boundaries, int32_t reps, double *graph_us, double *coop_us);

#ifdef __cplusplus
}
#endif
#endif /* LDPC_GB300_H */

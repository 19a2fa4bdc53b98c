// ldpc_decode_noalloc: the block-code decoder for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at decode time: code running inside a
// stream capture that must not add allocation nodes, real-time loops where a
// synchronous allocation would stall the pipeline, or hosts whose memory is
// fully reserved up front by another allocator.  For them the decoder's
// workspace lives in a fixed array compiled into this library (kNoallocBytes,
// 16 MiB, resident on every GPU that loads the library until the process
// exits).  The caller still passes its device input and output buffers.
//
// The array is a static __device__ object of this file.  In host code its name
// is only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress (on the first call made with that device
// current) and handed to the kernels as a plain pointer.
//
// Every call uses the same array, which keeps whatever the previous call left:
// the decode steps initialize everything they read (the flag words and the
// hard-decision words are cleared at the start of every decode, channel LLRs
// and messages are written before they are read).  Two calls whose GPU work
// overlaps -- on two streams, or from two threads -- use the same memory and
// race; serialize them.
#include "ldpc_internal.cuh"

#include <cstring>
#include <mutex>

namespace ldpc {

constexpr size_t kNoallocBytes = (size_t)16 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per device)
ldpc_status noalloc_base(void **out) {
    int dev = 0;
    LDPC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index %d out of range", dev);
        return LDPC_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LDPC_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

// bytes of scratch a decode of gamma frames of code d needs (same buffers as the
// allocating path, rounded to 256-byte boundaries)
static size_t noalloc_need(const QcDesc &d, size_t cap, size_t *off) {
    const size_t P32 = cap / 32;
    size_t o = 0;
    off[0] = o; o += align256((size_t)d.E * cap * 4);   // msg
    off[1] = o; o += align256((size_t)d.N * cap * 4);   // mu
    off[2] = o; o += align256((size_t)d.N * cap * 4);   // post
    off[3] = o; o += align256((size_t)d.N * P32 * 4);   // hw
    off[4] = o; o += align256(P32 * 5 * 4);             // flags
    off[5] = o; o += align256(cap * 2 * 4);             // iters, ok
    off[6] = o; o += align256(8 * sizeof(unsigned long long));  // counters
    off[7] = o; o += align256((P32 + 1) * sizeof(int)); // active-package list
    return o;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_decode_noalloc(ldpc_code c, const float *llr, int32_t gamma, const ldpc_decode_opts *opts,
                                float *post, uint8_t *hard, int32_t *iters, int32_t *ok, void *stream) {
    if (!c || !llr || gamma < 1 || !opts) {
        set_error("need code, llr, opts and gamma >= 1");
        return LDPC_EINVAL;
    }
    if (pointer_kind(llr) != 0 || (post && pointer_kind(post) != 0) || (hard && pointer_kind(hard) != 0) ||
        (iters && pointer_kind(iters) != 0) || (ok && pointer_kind(ok) != 0)) {
        set_error("ldpc_decode_noalloc takes device buffers only (host buffers would need staging memory)");
        return LDPC_EINVAL;
    }
    ldpc_status st = check_opts(c, opts);
    if (st != LDPC_OK) return st;
    if (opts->algo == LDPC_ALGO_NOMS) {
        set_error("ldpc_decode_noalloc supports sum-product and min-sum");
        return LDPC_EUNSUPPORTED;
    }
    const ldpc_decode_opts o = *opts;
    const size_t cap = ((size_t)gamma + 127) / 128 * 128;
    size_t off[8];
    const size_t need = noalloc_need(c->d, cap, off);
    if (need > kNoallocBytes) {
        set_error("ldpc_decode_noalloc: %d frames of this code need %zu bytes of scratch; the fixed scratch holds "
                  "%zu bytes (about %zu frames of this code)", gamma, need, kNoallocBytes,
                  (size_t)(128.0 * (double)kNoallocBytes / (double)noalloc_need(c->d, 128, off)));
        return LDPC_EINVAL;
    }
    void *base_v = nullptr;
    st = noalloc_base(&base_v);
    if (st != LDPC_OK) return st;
    noalloc_need(c->d, cap, off);
    unsigned char *base = (unsigned char *)base_v;
    // A private view of the code object whose workspace points into the scratch.  It
    // carries everything the decode steps read from a code: the QC description, and for
    // a general code the flag and the device index tables (which stay owned by c).  The
    // view is never passed to ldpc_code_destroy, the only place a workspace is freed.
    ldpc_code_s view;
    view.d = c->d;
    view.sparse = c->sparse;
    view.sp = c->sp;
    view.device = c->device;
    view.rate = c->rate;
    view.noms = nullptr;
    view.ws.gamma_cap = cap;
    view.ws.msg_bytes = (size_t)c->d.E * cap * 4;
    view.ws.msg = base + off[0];
    view.ws.mu = base + off[1];
    view.ws.post = (float *)(base + off[2]);
    view.ws.hw = (uint32_t *)(base + off[3]);
    view.ws.flags = (uint32_t *)(base + off[4]);
    view.ws.iters = (int32_t *)(base + off[5]);
    view.ws.counters = (unsigned long long *)(base + off[6]);
    view.ws.act = (int *)(base + off[7]);
    cudaStream_t s = (cudaStream_t)stream;
    st = qc_pack_llr(&view, llr, gamma, o, s);
    if (st != LDPC_OK) return st;
    st = qc_decode_device(&view, gamma, o, post != nullptr, s);
    if (st != LDPC_OK) return st;
    return qc_unpack_outputs(&view, gamma, o, post, hard, iters, ok, s);
}

}  // extern "C"

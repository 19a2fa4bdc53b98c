// Launch counting and per-launch event timing behind ldpc_profile_enable / ldpc_profile_read.
#include "ldpc_internal.cuh"

#include <cooperative_groups.h>

#include <atomic>
#include <vector>

namespace ldpc {

namespace {
std::atomic<long long> g_launches{0};
bool g_on = false;
struct Pair {
    cudaEvent_t a, b;
    int kind;
};
std::vector<Pair> g_pool;  // created events, reused across enable cycles
size_t g_used = 0;
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool profiling() { return g_on; }

int prof_begin(int kind, cudaStream_t s) {
    if (!g_on) return -1;
    if (g_used == g_pool.size()) {
        Pair p;
        if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        g_pool.push_back(p);
    }
    Pair &p = g_pool[g_used];
    p.kind = kind;
    cudaEventRecord(p.a, s);
    return (int)g_used++;
}

void prof_end(int slot, cudaStream_t s) {
    if (slot < 0) return;
    cudaEventRecord(g_pool[(size_t)slot].b, s);
}

// Bandwidth probe kernels: grid-stride sweeps over the buffer with four independent
// 16-byte loads in flight per thread.  mode 0 reads through L2 only (ld.global.cg, so
// an L2-resident buffer is served by L2, not L1), `sweeps` times within one launch (a
// sweep of an L2-sized buffer is too short to time against the launch), and folds the
// data into one word per thread block; mode 1 copies src to dst.
__global__ void __launch_bounds__(256) bw_read_kernel(const uint4 *__restrict__ src, size_t n16, int sweeps,
                                                     uint32_t *__restrict__ sink) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int r = 0; r < sweeps; ++r) {
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            uint4 a, b, c, d;
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w) : "l"(src + i));
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w) : "l"(src + i + stride));
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(c.x), "=r"(c.y), "=r"(c.z), "=r"(c.w) : "l"(src + i + 2 * stride));
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(d.x), "=r"(d.y), "=r"(d.z), "=r"(d.w) : "l"(src + i + 3 * stride));
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            uint4 a;
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w) : "l"(src + i));
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(sink + blockIdx.x, acc);
}

__global__ void __launch_bounds__(256) bw_copy_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                     size_t n16) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

ldpc_status ldpc_profile_enable(int32_t on) {
    g_on = on != 0;
    g_used = 0;
    g_launches.store(0);
    return LDPC_OK;
}

ldpc_status ldpc_profile_read(ldpc_profile *out) {
    if (!out) {
        set_error("out is NULL");
        return LDPC_EINVAL;
    }
    *out = ldpc_profile{};
    out->launches = g_launches.load();
    for (size_t i = 0; i < g_used; ++i) {
        Pair &p = g_pool[i];
        LDPC_CUDA_TRY(cudaEventSynchronize(p.b));
        float ms = 0.0f;
        LDPC_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.kind == 0) {
            out->cn_launches++;
            out->cn_ms += ms;
        } else {
            out->vn_launches++;
            out->vn_ms += ms;
        }
    }
    return LDPC_OK;
}

ldpc_status ldpc_bandwidth_probe(const void *src, void *dst, int64_t bytes, int32_t reps, int32_t mode,
                                 double *gbs_out, void *stream) {
    if (!src || !dst || !gbs_out || bytes < 16 || (bytes & 15) || reps < 1 || reps > 100000 ||
        (mode != 0 && mode != 1) || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15)) {
        set_error("need 16-byte aligned device src/dst, bytes a positive multiple of 16, 1 <= reps <= 100000, "
                  "mode 0 or 1, gbs_out");
        return LDPC_EINVAL;
    }
    if (pointer_kind(src) != 0 || pointer_kind(dst) != 0) {
        set_error("ldpc_bandwidth_probe takes device buffers");
        return LDPC_EINVAL;
    }
    if ((double)bytes * reps > 0x1p38) {  // keeps one probe to seconds
        set_error("bytes * reps must stay below 2^38");
        return LDPC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    LDPC_CUDA_TRY(cudaGetDevice(&dev));
    LDPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)sms * 8u;
    if (mode == 0 && (size_t)bytes < (size_t)blocks * 4u + 16u) {
        set_error("mode 0 needs dst to hold one word per block (%u blocks)", blocks);
        return LDPC_EINVAL;
    }
    const size_t n16 = (size_t)bytes / 16;
    cudaEvent_t a, b;
    LDPC_CUDA_TRY(cudaEventCreate(&a));
    LDPC_CUDA_TRY(cudaEventCreate(&b));
    // one untimed sweep (brings an L2-sized buffer into L2), then the timed ones: reads in one
    // launch, copies one launch per sweep
    count_launch();
    if (mode == 0) bw_read_kernel<<<blocks, 256, 0, s>>>((const uint4 *)src, n16, 1, (uint32_t *)dst);
    else bw_copy_kernel<<<blocks, 256, 0, s>>>((const uint4 *)src, (uint4 *)dst, n16);
    cudaEventRecord(a, s);
    if (mode == 0) {
        count_launch();
        bw_read_kernel<<<blocks, 256, 0, s>>>((const uint4 *)src, n16, reps, (uint32_t *)dst);
    } else {
        for (int r = 0; r < reps; ++r) {
            count_launch();
            bw_copy_kernel<<<blocks, 256, 0, s>>>((const uint4 *)src, (uint4 *)dst, n16);
        }
    }
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "bandwidth probe");
    const double moved = (double)bytes * reps * (mode == 1 ? 2.0 : 1.0);
    *gbs_out = ms > 0 ? moved / (ms * 1e-3) / 1e9 : 0.0;
    return LDPC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// phase-boundary probe: back-to-back launches replayed from a CUDA graph against
// grid-wide barriers inside one cooperative kernel, both with no work
// ---------------------------------------------------------------------------
namespace ldpc {
__global__ void __launch_bounds__(256) sync_empty_kernel(int *sink, int tag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) sink[0] = tag;
}

__global__ void __launch_bounds__(256) sync_coop_kernel(int *sink, int barriers) {
    cooperative_groups::grid_group g = cooperative_groups::this_grid();
    for (int i = 0; i < barriers; ++i) {
        if (threadIdx.x == 0 && blockIdx.x == 0) sink[0] = i;
        g.sync();
    }
}
}  // namespace ldpc

extern "C" ldpc_status ldpc_sync_probe(int32_t boundaries, int32_t reps, double *graph_us, double *coop_us) {
    if (boundaries < 1 || boundaries > 4096 || reps < 1 || reps > 10000 || !graph_us || !coop_us) {
        set_error("need 1 <= boundaries <= 4096, 1 <= reps <= 10000, graph_us, coop_us");
        return LDPC_EINVAL;
    }
    int dev = 0, sms = 1, coop = 0, per_sm = 0;
    LDPC_CUDA_TRY(cudaGetDevice(&dev));
    LDPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    LDPC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sync_coop_kernel, 256, 0));
    if (!coop || per_sm < 1) {
        set_error("cooperative launch unavailable on this device");
        return LDPC_EUNSUPPORTED;
    }
    // two resident blocks per SM at most (the batch's check pass), all of them resident
    const int cblocks = sms * (per_sm < 2 ? per_sm : 2);
    int *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    // one phase per boundary, with the batch's grid sizes in turn: tile rebuild, syndrome,
    // check pass, variable pass
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        static const int mult[4] = {1, 4, 2, 3};
        for (int i = 0; i < boundaries; ++i) sync_empty_kernel<<<sms * mult[i & 3], 256, 0, s>>>(sink, i);
        e = cudaStreamEndCapture(s, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    float ms_graph = 0.0f, ms_coop = 0.0f;
    if (e == cudaSuccess) {
        for (int w = 0; w < 3 && e == cudaSuccess; ++w) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_graph, a, b);
        count_launch((long long)(reps + 3) * boundaries);
    }
    if (e == cudaSuccess) {
        int nb = boundaries;
        void *args[] = {&sink, &nb};
        for (int w = 0; w < 3 && e == cudaSuccess; ++w)
            e = cudaLaunchCooperativeKernel((const void *)sync_coop_kernel, cblocks, 256, args, 0, s);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = cudaLaunchCooperativeKernel((const void *)sync_coop_kernel, cblocks, 256, args, 0, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_coop, a, b);
        count_launch(reps + 3);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "phase-boundary probe");
    *graph_us = 1e3 * ms_graph / reps / boundaries;
    *coop_us = 1e3 * ms_coop / reps / boundaries;
    return LDPC_OK;
}

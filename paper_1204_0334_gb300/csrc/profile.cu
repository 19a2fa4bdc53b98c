// Launch counting and per-launch event timing behind ldpc_profile_enable / ldpc_profile_read.
#include "ldpc_internal.cuh"

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

}  // extern "C"

// Continuous Monte-Carlo simulation (the protocol of Sec. V) with frame slots
// that are refilled as soon as their frame stops.
//
// Decoding gamma frames to the end before drawing the next gamma wastes most of
// the early-stopping gain: a package of 32 frames keeps being visited until its
// slowest frame stops, and the whole batch waits for the slowest package.
// Here every lane of the package layout is a frame slot.  One step of the
// simulation is
//
//   syndrome: of every slot's decisions so far (eq. (hrddcs))
//   retire:   a frame whose decisions after a >= 1 iterations satisfy every
//             check (C-11 stopping), or that has run max_iter iterations,
//             leaves its slot; the next frame id takes the slot
//   compact:  the packages with a running or retiring frame
//   channel:  the new frames' channel LLRs (Philox + Box-Muller with the
//             counter of ldpc_channel) into the slots' channel store
//   check pass: one iteration of every running frame; a new frame's
//             outgoing messages are set to 0
//   variable pass: one iteration of every running frame (a new frame gets
//             beta = mu + 0 = mu, the initialization of Alg. 1, and its
//             first check pass comes in the next step); it also counts a
//             retired frame's wrong bits from its last decisions before the
//             new frame's overwrite them
//
// so each frame runs exactly the iterations the batch decoder gives it, with
// the same decisions, while the slots stay busy.  The retire
// kernel of the next step adds the retired frames' counts to the totals.  Frame ids are
// handed out in order from a device counter, so the frames simulated are
// always first_frame .. first_frame + frames - 1 (the set does not depend on
// which slot a frame lands in).  Once the frame-error target is met no new
// frame starts and the frames in flight finish.
#include "qc_device.cuh"

#include <chrono>
#include <cstring>

struct ldpc_sim_state {
    size_t slots = 0;
    uint32_t *sflags = nullptr;           // [P][2V]: retire[V], refill[V]
    uint64_t *fid = nullptr;              // [slots] frame id of the slot's frame
    int *errs = nullptr;                  // [slots] wrong bits of the frame retired last step
    int *age = nullptr;                   // [slots] iterations completed by the slot's frame
    int *pend = nullptr;                  // [slots] 2 * iterations + ok of the frame retired last step, or -1
    void *mu = nullptr;                   // channel LLRs, frame-major [slots][N rounded up to 4]
    size_t mu_bytes = 0;
    int *rlist = nullptr;                 // [slots] slots refilled this step
    int *rcount = nullptr;                // [2] entries of rlist, by step parity
    unsigned long long *next = nullptr;   // next frame index to hand out
    unsigned long long *host = nullptr;   // pinned [2][16]: counters, active packages
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace ldpc {

void sim_free(ldpc_sim_state *st) {
    if (!st) return;
    cudaFree(st->sflags);
    cudaFree(st->fid);
    cudaFree(st->errs);
    cudaFree(st->age);
    cudaFree(st->pend);
    cudaFree(st->mu);
    cudaFree(st->rlist);
    cudaFree(st->rcount);
    cudaFree(st->next);
    if (st->host) cudaFreeHost(st->host);
    for (auto &e : st->ev)
        if (e) cudaEventDestroy(e);
    delete st;
}

namespace {

ldpc_status sim_ensure(ldpc_code c, size_t slots) {
    ldpc_sim_state *&st = c->sim;
    const size_t mu_bytes = slots * (size_t)((c->d.N + 3) & ~3) * 4;
    if (st && st->slots >= slots && st->mu_bytes >= mu_bytes) return LDPC_OK;
    LDPC_CUDA_TRY(cudaDeviceSynchronize());
    sim_free(st);
    st = new ldpc_sim_state();
    const size_t words = slots / 32 * 2;  // 2 words per 32 slots, any V
    if (cudaMalloc(&st->sflags, words * 4) != cudaSuccess || cudaMalloc(&st->fid, slots * 8) != cudaSuccess ||
        cudaMalloc(&st->errs, slots * 4) != cudaSuccess || cudaMalloc(&st->age, slots * 4) != cudaSuccess ||
        cudaMalloc(&st->pend, slots * 4) != cudaSuccess || cudaMalloc(&st->next, 8) != cudaSuccess ||
        cudaMalloc(&st->rlist, slots * 4) != cudaSuccess || cudaMalloc(&st->rcount, 2 * 4) != cudaSuccess ||
        cudaMalloc(&st->mu, mu_bytes) != cudaSuccess ||
        cudaHostAlloc(&st->host, 2 * 16 * 8, cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        sim_free(st);
        st = nullptr;
        set_error("device allocation for %zu simulation slots failed", slots);
        return LDPC_ENOMEM;
    }
    st->slots = slots;
    st->mu_bytes = mu_bytes;
    return LDPC_OK;
}

}  // namespace

// every slot empty, nothing pending, counters zero
__global__ void sim_init_kernel(uint32_t *flags, int *errs, int *age, int *pend, unsigned long long *next,
                                int *rcount, unsigned long long *counters, int P, int V) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int slots = P * 32 * V;
    if (i < slots) {
        errs[i] = 0;
        age[i] = 0;
        pend[i] = -1;
    }
    if (i < P * 5 * V) {
        const int q = i % (5 * V);
        flags[i] = q < V ? 0xffffffffu : 0u;  // done words: the slot holds no running frame
    }
    if (i < 8) counters[i] = 0ull;
    if (i == 0) *next = 0ull;
    if (i < 2) rcount[i] = 0;
}

// One warp per (package, word v); lane = slot.  Tallies the frames retired by
// the previous step, retires the frames that stop now and refills slots.
__global__ void sim_retire_kernel(uint32_t *__restrict__ flags, uint32_t *__restrict__ sflags,
                                  uint64_t *__restrict__ fid, int *__restrict__ errs, int *__restrict__ age,
                                  int *__restrict__ pend, unsigned long long *__restrict__ next,
                                  int *__restrict__ rlist, int *__restrict__ rcount,
                                  unsigned long long *counters, int P, int V, int max_iter, int early_stop,
                                  unsigned long long first_frame, unsigned long long limit,
                                  unsigned long long target, int parity) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw == 0 && lane == 0) rcount[parity ^ 1] = 0;  // the next step's list
    if (gw >= P * V) return;  // warp-uniform
    const int pk = gw / V, v = gw - pk * V;
    const size_t slot = (size_t)pk * 32 * V + lane * V + v;
    uint32_t *F = flags + (size_t)pk * 5 * V;
    const uint32_t D = F[v], U = F[V + v];

    // frames retired by the previous step: their wrong bits were counted by its variable pass
    const int pr = pend[slot];
    unsigned long long fr = 0, fe = 0, be = 0, is = 0, ud = 0;
    if (pr >= 0) {
        const int e = errs[slot];
        errs[slot] = 0;
        pend[slot] = -1;
        fr = 1;
        be = (unsigned long long)e;
        fe = e > 0;
        is = (unsigned long long)(pr >> 1);
        ud = (e > 0 && (pr & 1)) ? 1 : 0;
    }
    if (__ballot_sync(0xffffffffu, pr >= 0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fr += __shfl_xor_sync(0xffffffffu, fr, o);
            fe += __shfl_xor_sync(0xffffffffu, fe, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            is += __shfl_xor_sync(0xffffffffu, is, o);
            ud += __shfl_xor_sync(0xffffffffu, ud, o);
        }
        if (lane == 0) {
            atomicAdd(counters + 0, fr);
            if (fe) atomicAdd(counters + 1, fe);
            if (be) atomicAdd(counters + 2, be);
            atomicAdd(counters + 3, is);
            if (ud) atomicAdd(counters + 4, ud);
        }
    }

    // the check pass just computed the syndrome of the decisions after a iterations
    const bool running = !((D >> lane) & 1u);
    int a = age[slot];
    const bool sat = !((U >> lane) & 1u);
    const bool ret = running && ((early_stop && a >= 1 && sat) || a >= max_iter);
    if (ret) pend[slot] = 2 * a + (sat ? 1 : 0);

    // refill: no new frame once the frame-error target is met (read from earlier steps' totals)
    const bool stop = *(volatile unsigned long long *)(counters + 1) >= target;
    const uint32_t want = __ballot_sync(0xffffffffu, (!running || ret) && !stop);
    unsigned long long base = 0;
    if (want) {
        if (lane == 0) base = atomicAdd(next, (unsigned long long)__popc(want));
        base = __shfl_sync(0xffffffffu, base, 0);
    }
    const unsigned long long idx = base + (unsigned long long)__popc(want & ((1u << lane) - 1u));
    const bool fill = ((want >> lane) & 1u) && idx < limit;
    // iterations completed at the next step's retire kernel (a new frame's first step only
    // initializes its messages)
    if (fill) {
        fid[slot] = first_frame + idx;
        a = 0;
    } else if (running && !ret) {
        a += 1;
    }
    age[slot] = a;
    const uint32_t retw = __ballot_sync(0xffffffffu, ret);
    const uint32_t fillw = __ballot_sync(0xffffffffu, fill);
    if (fillw) {
        int rb = 0;
        if (lane == 0) rb = atomicAdd(rcount + parity, __popc(fillw));
        rb = __shfl_sync(0xffffffffu, rb, 0);
        if (fill) rlist[rb + __popc(fillw & ((1u << lane) - 1u))] = (int)slot;
    }
    if (lane == 0) {
        F[v] = (D | retw) & ~fillw;
        F[V + v] = 0u;  // set again by the next check pass
        sflags[(size_t)pk * 2 * V + v] = retw;
        sflags[(size_t)pk * 2 * V + V + v] = fillw;
    }
}

// Channel LLRs of the frames that entered a slot this step, frame-major
// ([slot][N4], N4 = N rounded up to 4): clipped floats, or int8 quantized with
// qscale (as the batch path's channel kernel rounds them).  Consecutive threads
// take consecutive groups of 4 bits of one frame, so each warp writes whole lines.
template <bool I8>
__global__ void sim_channel_kernel(void *__restrict__ mu, const int *__restrict__ rlist,
                                   const int *__restrict__ rcount, const uint64_t *__restrict__ fid, int N,
                                   int parity, uint64_t seed, float sigma, float s2, float clip, float qscale) {
    const int cnt = rcount[parity];
    if (cnt == 0) return;
    const int Q = (N + 3) / 4;
    const size_t N4 = (size_t)Q * 4;
    const long long total = (long long)cnt * Q;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / Q);
        const int q = (int)(i - (long long)r * Q);
        const int slot = rlist[r];
        float x[4];
        channel_quad(seed, fid[slot], q, sigma, s2, x);
        if (I8) {
            uint32_t w = 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float v = fminf(fmaxf(rintf(x[e] * qscale), -127.0f), 127.0f);
                w |= (uint32_t)(uint8_t)(int8_t)v << (8 * e);
            }
            reinterpret_cast<uint32_t *>(mu)[((size_t)slot * N4 + 4 * q) / 4] = w;
        } else {
            reinterpret_cast<float4 *>(mu)[((size_t)slot * N4 + 4 * q) / 4] =
                make_float4(clipf(x[0], clip), clipf(x[1], clip), clipf(x[2], clip), clipf(x[3], clip));
        }
    }
}

// Runs the continuous simulation; h receives counters[0..4] (frames, frame
// errors, bit errors, iterations, undetected).
ldpc_status qc_ber_sim_refill(ldpc_code c, double sigma, uint64_t seed, uint64_t first_frame, int64_t max_frames,
                              int64_t target, int gamma, const ldpc_decode_opts &o, unsigned long long *h,
                              cudaStream_t s) {
    const int V = lanes_per_word(o.msg), W = 32 * V;
    const int P = (gamma + W - 1) / W;
    const size_t slots = (size_t)P * W;
    ldpc_status st = qc_ensure_workspace(c, slots, 0);
    if (st != LDPC_OK) return st;
    st = sim_ensure(c, c->ws.gamma_cap);
    if (st != LDPC_OK) return st;
    ldpc_sim_state *S = c->sim;
    {
        const int n = (int)(slots > (size_t)P * 5 * V ? slots : (size_t)P * 5 * V);
        sim_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->ws.flags, S->errs, S->age, S->pend, S->next,
                                                        S->rcount, c->ws.counters, P, V);
        count_launch();
    }
    RefillArgs rf;
    rf.sflags = S->sflags;
    rf.errs = S->errs;
    rf.mu = S->mu;
    const float fsig = (float)sigma, s2 = (float)(2.0 / (sigma * sigma));
    const bool i8 = o.algo == LDPC_ALGO_MS;
    int sms = 0, dev = 0;
    LDPC_CUDA_TRY(cudaGetDevice(&dev));
    LDPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int cblocks = (sms > 0 ? sms : 1) * 8;
    int parity = 0;
    const unsigned long long limit = (unsigned long long)max_frames;
    const unsigned long long tgt = target < 0 ? 0ull : (unsigned long long)target;
    const int rblocks = (P * V * 32 + 255) / 256;

    auto step = [&]() -> ldpc_status {
        ldpc_status e = qc_syndrome(c, P, V, V, s);  // unsat words
        if (e != LDPC_OK) return e;
        sim_retire_kernel<<<rblocks, 256, 0, s>>>(c->ws.flags, S->sflags, S->fid, S->errs, S->age, S->pend, S->next,
                                                  S->rlist, S->rcount, c->ws.counters, P, V, o.max_iter,
                                                  o.early_stop, first_frame, limit, tgt, parity);
        e = qc_compact(c, P, V, s, S->sflags);
        if (e != LDPC_OK) return e;
        if (i8)
            sim_channel_kernel<true><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N, parity, seed,
                                                             fsig, s2, 1e30f, ldexpf(1.0f, o.frac_bits));
        else
            sim_channel_kernel<false><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N, parity,
                                                              seed, fsig, s2, o.clip, 1.0f);
        parity ^= 1;
        const int slot_cn = prof_begin(0, s);
        e = qc_cn_pipe(c, o, 1, s, S->sflags, o.algo == LDPC_ALGO_NOMS ? S->age : nullptr);
        if (e != LDPC_OK) return e;
        prof_end(slot_cn, s);
        const int slot_vn = prof_begin(1, s);
        e = qc_vn_refill(c, o, rf, s);
        if (e != LDPC_OK) return e;
        prof_end(slot_vn, s);
        count_launch(6);
        return LDPC_OK;
    };

    // Steps are queued in chunks; after each chunk the totals and the number of
    // active packages are copied to pinned memory and the previous chunk's copy
    // is read, so the device always has a chunk queued while the host checks.
    // The loop ends when a chunk ends with no active package (every started
    // frame has retired and been counted).
    constexpr int kChunk = 2;
    const int64_t max_steps = ((int64_t)(max_frames / (int64_t)slots) + 2) * (int64_t)(o.max_iter + 2) + 16;
    int64_t steps = 0;
    int b = 0;
    bool have_prev = false;
    for (;;) {
        for (int i = 0; i < kChunk; ++i) {
            st = step();
            if (st != LDPC_OK) return st;
        }
        steps += kChunk;
        unsigned long long *hb = S->host + 16 * b;
        LDPC_CUDA_TRY(cudaMemcpyAsync(hb, c->ws.counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LDPC_CUDA_TRY(cudaMemcpyAsync(hb + 8, c->ws.act, sizeof(int), cudaMemcpyDeviceToHost, s));
        LDPC_CUDA_TRY(cudaEventRecord(S->ev[b], s));
        if (have_prev) {
            LDPC_CUDA_TRY(cudaEventSynchronize(S->ev[b ^ 1]));
            const unsigned long long *hp = S->host + 16 * (b ^ 1);
            int active = 0;
            std::memcpy(&active, hp + 8, sizeof(int));
            if (active == 0) break;
        }
        have_prev = true;
        b ^= 1;
        if (steps > max_steps) {
            set_error("continuous simulation did not drain after %lld steps", (long long)steps);
            return LDPC_ETIMEOUT;
        }
    }
    LDPC_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(h, S->host + 16 * (b ^ 1), 8 * sizeof(unsigned long long));
    return LDPC_OK;
}

}  // namespace ldpc

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
//   retire:   a frame whose decisions after a >= 1 complete iterations satisfy
//             every check, or that has run max_iter iterations, leaves its
//             slot; the next frame id takes the slot
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
//
// With random codewords (encode.cu) the step also counts the retiring frames'
// wrong information bits against their codewords (right after the check, from
// the decisions the variable pass would otherwise count) and encodes the new
// frames' codewords before the channel sends them.
#include "qc_device.cuh"

#include <chrono>
#include <cstring>

struct ldpc_sim_state {
    size_t slots = 0;
    uint32_t *sflags = nullptr;           // [P][2V]: retire[V], refill[V]
    uint64_t *fid = nullptr;              // [slots] frame id of the slot's frame
    uint64_t *rfid = nullptr;             // [slots] frame id of the frame that retired from the slot this step
    int *errs = nullptr;                  // [slots] wrong bits of the frame retired last step
    int *age = nullptr;                   // [slots] iterations completed by the slot's frame
    int *pend = nullptr;                  // [slots] 2 * iterations + ok of the frame retired last step, or -1
    void *mu = nullptr;                   // channel LLRs, frame-major [slots][N rounded up to 4]
    size_t mu_bytes = 0;
    int *rlist = nullptr;                 // [slots] slots refilled this step
    int *rcount = nullptr;                // [2] entries of rlist, by step parity
    uint32_t *cwf = nullptr;              // random codewords: [slots][ceil(N / 32)] the slot's codeword bits
    size_t cwf_slots = 0;
    unsigned int *tickets = nullptr;      // [P + 1]: finished blocks per package, finished packages
    unsigned long long *next = nullptr;   // next frame index to hand out
    unsigned long long *host = nullptr;   // pinned [2][16]: counters, active packages
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace ldpc {

void sim_free(ldpc_sim_state *st) {
    if (!st) return;
    cudaFree(st->sflags);
    cudaFree(st->fid);
    cudaFree(st->rfid);
    cudaFree(st->errs);
    cudaFree(st->age);
    cudaFree(st->pend);
    cudaFree(st->mu);
    cudaFree(st->rlist);
    cudaFree(st->rcount);
    cudaFree(st->cwf);
    cudaFree(st->tickets);
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
        cudaMalloc(&st->rfid, slots * 8) != cudaSuccess ||
        cudaMalloc(&st->errs, slots * 4) != cudaSuccess || cudaMalloc(&st->age, slots * 4) != cudaSuccess ||
        cudaMalloc(&st->pend, slots * 4) != cudaSuccess || cudaMalloc(&st->next, 8) != cudaSuccess ||
        cudaMalloc(&st->rlist, slots * 4) != cudaSuccess || cudaMalloc(&st->rcount, 2 * 4) != cudaSuccess ||
        cudaMalloc(&st->tickets, (slots / 32 + 2) * 4) != cudaSuccess ||
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
                                int *rcount, unsigned int *tickets, unsigned long long *counters, int P, int V) {
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
    if (i <= P) tickets[i] = 0u;
}

// arguments of the step's check kernel
struct SimArgs {
    const uint32_t *hw;
    uint32_t *flags, *sflags;
    uint64_t *fid, *rfid;
    int *errs, *age, *pend;
    unsigned long long *next, *counters;
    int *rlist, *rcount, *act;
    unsigned int *tickets;  // [P]: finished syndrome blocks per package; [P]: finished packages
    int P, max_iter, early_stop, parity;
    unsigned long long first_frame, limit, target;
};

// One warp per (package, word v); lane = slot.  Tallies the frames retired by the
// previous step, retires the frames that stop now and refills slots.  Flag words written
// by other blocks of this launch are read past L1.
template <int V>
__device__ void retire_word(const SimArgs &sa, int pk, int v, int lane) {
    const size_t slot = (size_t)pk * 32 * V + lane * V + v;
    uint32_t *F = sa.flags + (size_t)pk * 5 * V;
    const uint32_t D = __ldcg(F + v), U = __ldcg(F + V + v);

    // frames retired by the previous step: their wrong bits were counted by its variable pass
    const int pr = sa.pend[slot];
    unsigned long long fr = 0, fe = 0, be = 0, is = 0, ud = 0, b2 = 0;
    if (pr >= 0) {
        const int e = sa.errs[slot];
        sa.errs[slot] = 0;
        sa.pend[slot] = -1;
        fr = 1;
        be = (unsigned long long)e;
        b2 = be * be;
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
            b2 += __shfl_xor_sync(0xffffffffu, b2, o);
        }
        if (lane == 0) {
            atomicAdd(sa.counters + 0, fr);
            if (fe) atomicAdd(sa.counters + 1, fe);
            if (be) atomicAdd(sa.counters + 2, be);
            atomicAdd(sa.counters + 3, is);
            if (ud) atomicAdd(sa.counters + 4, ud);
            if (b2) atomicAdd(sa.counters + 5, b2);
        }
    }

    // the syndrome of the decisions after a iterations was just computed
    const bool running = !((D >> lane) & 1u);
    int a = sa.age[slot];
    const bool sat = !((U >> lane) & 1u);
    const bool ret = running && ((sa.early_stop && a >= 1 && sat) || a >= sa.max_iter);
    if (ret) {
        sa.pend[slot] = 2 * a + (sat ? 1 : 0);
        sa.rfid[slot] = sa.fid[slot];
    }

    // refill: no new frame once the frame-error target is met (read from earlier totals)
    const bool stop = *(volatile unsigned long long *)(sa.counters + 1) >= sa.target;
    const uint32_t want = __ballot_sync(0xffffffffu, (!running || ret) && !stop);
    unsigned long long base = 0;
    if (want) {
        if (lane == 0) base = atomicAdd(sa.next, (unsigned long long)__popc(want));
        base = __shfl_sync(0xffffffffu, base, 0);
    }
    const unsigned long long idx = base + (unsigned long long)__popc(want & ((1u << lane) - 1u));
    const bool fill = ((want >> lane) & 1u) && idx < sa.limit;
    // iterations completed at the next step's check (a new frame's first step only
    // initializes its messages)
    if (fill) {
        sa.fid[slot] = sa.first_frame + idx;
        a = 0;
    } else if (running && !ret) {
        a += 1;
    }
    sa.age[slot] = a;
    const uint32_t retw = __ballot_sync(0xffffffffu, ret);
    const uint32_t fillw = __ballot_sync(0xffffffffu, fill);
    if (fillw) {
        int rb = 0;
        if (lane == 0) rb = atomicAdd(sa.rcount + sa.parity, __popc(fillw));
        rb = __shfl_sync(0xffffffffu, rb, 0);
        if (fill) sa.rlist[rb + __popc(fillw & ((1u << lane) - 1u))] = (int)slot;
    }
    if (lane == 0) {
        F[v] = (D | retw) & ~fillw;
        F[V + v] = 0u;  // set again by the next syndrome
        sa.sflags[(size_t)pk * 2 * V + v] = retw;
        sa.sflags[(size_t)pk * 2 * V + V + v] = fillw;
    }
}

// The step's check kernel: hard-decision syndrome (eq. hrddcs), per-frame stop and refill,
// and the list of active packages, in one launch.  Block (x, pk) checks rows 256x ..
// 256x + 255 of package pk against the packed decisions and ORs the unsatisfied frames
// into the package's unsat words; the last block to finish a package (atomic ticket after
// a fence) retires and refills that package's slots; the last package to finish lists the
// packages with a running or retiring frame (act[0] = count, act[1..]) for the passes.
// Nothing waits: a block either continues with the later stage or returns.
template <int V>
__global__ void __launch_bounds__(256) sim_check_kernel(const QcDesc d, SimArgs sa) {
    __shared__ int s_last;
    __shared__ int s_wsum[8];
    __shared__ int s_base;
    const int pk = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const int m = blockIdx.x * blockDim.x + threadIdx.x;
        uint32_t syn[V];
#pragma unroll
        for (int v = 0; v < V; ++v) syn[v] = 0u;
        if (m < d.M) {
            const int j = (int)fdiv((uint32_t)m, d.divP), r = m - j * d.p;
            for (int l = 0; l < d.L; ++l) {
                const int a = d.shift[j * d.L + l];
                if (a < 0) continue;
                int k = r + a;
                if (k >= d.p) k -= d.p;
                const uint32_t *h = sa.hw + ((size_t)pk * d.N + (size_t)l * d.p + k) * V;
#pragma unroll
                for (int v = 0; v < V; ++v) syn[v] ^= h[v];
            }
        }
        uint32_t *unsat = sa.flags + (size_t)pk * 5 * V + V;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t any = __reduce_or_sync(0xffffffffu, syn[v]);
            if (any && lane == 0) atomicOr(unsat + v, any);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(sa.tickets + pk, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (warp < V) retire_word<V>(sa, pk, warp, lane);
    if (threadIdx.x == 0) sa.tickets[pk] = 0u;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(sa.tickets + sa.P, 1u) == (unsigned)sa.P - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // compaction over all packages
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int p0 = 0; p0 < sa.P; p0 += blockDim.x) {
        const int q = p0 + threadIdx.x;
        bool on = false;
        if (q < sa.P)
            for (int v = 0; v < V; ++v)
                on |= (~__ldcg(sa.flags + (size_t)q * 5 * V + v) | __ldcg(sa.sflags + (size_t)q * 2 * V + v)) != 0u;
        const uint32_t bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) s_wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += s_wsum[w];
            all += s_wsum[w];
        }
        const int base = s_base;
        if (on) sa.act[1 + base + before + __popc(bal & ((1u << lane) - 1u))] = q;
        __syncthreads();
        if (threadIdx.x == 0) s_base = base + all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sa.act[0] = s_base;
        sa.rcount[sa.parity ^ 1] = 0;  // the next step's list of new frames
        sa.tickets[sa.P] = 0u;
    }
}

// Channel LLRs of the frames that entered a slot this step, frame-major
// ([slot][N4], N4 = N rounded up to 4): clipped floats, or int8 quantized with
// qscale (as the batch path's channel kernel rounds them).  Consecutive threads
// take consecutive groups of 4 bits of one frame, so each warp writes whole lines.
// CW: the slot's codeword (row cwf[slot][NW]) is sent, else the all-zero word.
template <bool I8, bool CW>
__global__ void sim_channel_kernel(void *__restrict__ mu, const int *__restrict__ rlist,
                                   const int *__restrict__ rcount, const uint64_t *__restrict__ fid, int N,
                                   int parity, uint64_t seed, float sigma, float s2, float clip, float qscale,
                                   const uint32_t *__restrict__ cwf, int NW) {
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
        const uint32_t bits = CW ? (cwf[(size_t)slot * NW + (q >> 3)] >> (4 * (q & 7))) & 15u : 0u;
        channel_quad(seed, fid[slot], q, sigma, s2, x, bits);
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

// Streaming decode of a caller's batch (ldpc_decode): the frames that entered a slot
// this step copy their channel LLRs from row fid of the caller's [gamma][N] buffer
// (device memory, or pinned host memory read through its device mapping) into the
// slots' frame-major store: clipped for sum-product, quantized for min-sum exactly as
// the batch path's packing does.
// VEC: rows start on 16-byte boundaries (N a multiple of 4, llr 16-byte aligned), so each thread
// reads its 4 values with one 16-byte load (a warp reads 512 contiguous bytes of the row)
template <bool I8, bool VEC>
__global__ void stream_load_kernel(const float *__restrict__ llr, void *__restrict__ mu,
                                   const int *__restrict__ rlist, const int *__restrict__ rcount,
                                   const uint64_t *__restrict__ fid, int N, int parity, float clip, float qscale) {
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
        const float *row = llr + (size_t)fid[slot] * N;
        float x[4];
        if (VEC) {
            const float4 v4 = reinterpret_cast<const float4 *>(row)[q];
            x[0] = v4.x, x[1] = v4.y, x[2] = v4.z, x[3] = v4.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = 4 * q + e < N ? row[4 * q + e] : 0.0f;
        }
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

// Streaming decode: the outputs of the frames that retired this step, written before the
// step's passes overwrite their slots -- hard decisions (row fid of the caller's
// [gamma][N] bytes, from the slots' packed decision words), iteration count and ok flag.
// Block (package, word v); threads over the variables.  VEC: rows of hard start on 4-byte
// boundaries (N a multiple of 4, hard 4-byte aligned), so each thread writes 4 decisions at once.
template <bool VEC>
__global__ void __launch_bounds__(256)
stream_out_kernel(const uint32_t *__restrict__ hw, const uint32_t *__restrict__ sflags, const uint64_t *__restrict__ rfid,
                  const int *__restrict__ pend, uint8_t *__restrict__ hard, int32_t *__restrict__ iters,
                  int32_t *__restrict__ ok, int N, int V) {
    const int pk = blockIdx.x, v = blockIdx.y;
    const uint32_t R = sflags[(size_t)pk * 2 * V + v];  // retire word
    if (R == 0u) return;
    if (threadIdx.x < 32 && ((R >> threadIdx.x) & 1u)) {
        const size_t slot = (size_t)pk * 32 * V + threadIdx.x * V + v;
        const uint64_t f = rfid[slot];
        const int pr = pend[slot];
        if (iters) iters[f] = pr >> 1;
        if (ok) ok[f] = pr & 1;
    }
    if (!hard) return;
    if constexpr (VEC) {
        for (int n4 = threadIdx.x; 4 * n4 < N; n4 += blockDim.x) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) w[e] = hw[((size_t)pk * N + 4 * n4 + e) * V + v];
            for (uint32_t b = R; b; b &= b - 1) {
                const int ln = __ffs(b) - 1;
                const uint64_t f = rfid[(size_t)pk * 32 * V + ln * V + v];
                uint32_t out = 0u;
#pragma unroll
                for (int e = 0; e < 4; ++e) out |= ((w[e] >> ln) & 1u) << (8 * e);
                reinterpret_cast<uint32_t *>(hard + f * (uint64_t)N)[n4] = out;
            }
        }
    } else {
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const uint32_t w = hw[((size_t)pk * N + n) * V + v];
            for (uint32_t b = R; b; b &= b - 1) {
                const int ln = __ffs(b) - 1;
                const uint64_t f = rfid[(size_t)pk * 32 * V + ln * V + v];
                hard[f * (uint64_t)N + n] = (uint8_t)((w >> ln) & 1u);
            }
        }
    }
}

// Runs the continuous simulation; h receives counters[0..5] (frames, frame
// errors, bit errors, iterations, undetected, sum over frames of the squared
// bit-error count).
// With io (streaming decode of a caller's batch): frames 0 .. max_frames - 1 are the rows of
// io->llr, each frame's outputs go to io->hard / iters / ok as it retires, and no errors are
// counted (sigma, seed, first_frame and target are unused).
ldpc_status qc_ber_sim_refill(ldpc_code c, double sigma, uint64_t seed, uint64_t first_frame, int64_t max_frames,
                              int64_t target, int gamma, const ldpc_decode_opts &o, unsigned long long *h,
                              cudaStream_t s, const StreamIO *io) {
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
                                                        S->rcount, S->tickets, c->ws.counters, P, V);
        count_launch();
    }
    // random codewords: the encoder and each slot's codeword row
    const bool cw = !io && o.codewords == LDPC_CODEWORDS_RANDOM;
    if (io) {
        first_frame = 0;
        target = (int64_t)1 << 62;
    }
    const int NW = enc_words(c);
    if (cw) {
        st = enc_ensure_device(c, slots / 32);
        if (st != LDPC_OK) return st;
        if (S->cwf_slots < slots) {
            LDPC_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(S->cwf);
            S->cwf = nullptr;
            S->cwf_slots = 0;
            if (cudaMalloc(&S->cwf, slots * (size_t)NW * 4) != cudaSuccess) {
                cudaGetLastError();
                S->cwf = nullptr;
                set_error("device allocation of %zu codeword rows failed", slots);
                return LDPC_ENOMEM;
            }
            S->cwf_slots = slots;
        }
    }
    RefillArgs rf;
    rf.sflags = S->sflags;
    rf.errs = (cw || io) ? nullptr : S->errs;  // with codewords the errors are counted against them
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

    SimArgs sa;
    sa.hw = c->ws.hw;
    sa.flags = c->ws.flags;
    sa.sflags = S->sflags;
    sa.fid = S->fid;
    sa.rfid = S->rfid;
    sa.errs = S->errs;
    sa.age = S->age;
    sa.pend = S->pend;
    sa.next = S->next;
    sa.counters = c->ws.counters;
    sa.rlist = S->rlist;
    sa.rcount = S->rcount;
    sa.act = c->ws.act;
    sa.tickets = S->tickets;
    sa.P = P;
    sa.max_iter = o.max_iter;
    sa.early_stop = o.early_stop;
    sa.first_frame = first_frame;
    sa.limit = limit;
    sa.target = tgt;
    const dim3 cgrd((c->d.M + 255) / 256, P);

    auto step = [&]() -> ldpc_status {
        sa.parity = parity;
        if (V == 1) sim_check_kernel<1><<<cgrd, 256, 0, s>>>(c->d, sa);
        else if (V == 2) sim_check_kernel<2><<<cgrd, 256, 0, s>>>(c->d, sa);
        else sim_check_kernel<4><<<cgrd, 256, 0, s>>>(c->d, sa);
        ldpc_status e = LDPC_OK;
        if (io) {
            // the retiring frames' outputs, then the new frames' channel LLRs from the caller's rows
            const bool vin = (c->d.N % 4) == 0 && ((uintptr_t)io->llr & 15u) == 0;
            const bool vout = (c->d.N % 4) == 0 && ((uintptr_t)io->hard & 3u) == 0;
            if (vout)
                stream_out_kernel<true><<<dim3(P, V), 256, 0, s>>>(c->ws.hw, S->sflags, S->rfid, S->pend, io->hard,
                                                                   io->iters, io->ok, c->d.N, V);
            else
                stream_out_kernel<false><<<dim3(P, V), 256, 0, s>>>(c->ws.hw, S->sflags, S->rfid, S->pend, io->hard,
                                                                    io->iters, io->ok, c->d.N, V);
            auto load = [&](auto kfn, float clip, float qs) {
                kfn<<<cblocks, 256, 0, s>>>(io->llr, S->mu, S->rlist, S->rcount, S->fid, c->d.N, parity, clip, qs);
            };
            if (i8) {
                if (vin) load(stream_load_kernel<true, true>, 1e30f, ldexpf(1.0f, o.frac_bits));
                else load(stream_load_kernel<true, false>, 1e30f, ldexpf(1.0f, o.frac_bits));
            } else {
                if (vin) load(stream_load_kernel<false, true>, o.clip, 1.0f);
                else load(stream_load_kernel<false, false>, o.clip, 1.0f);
            }
            count_launch(2);
            parity ^= 1;
            const int slot_cn = prof_begin(0, s);
            e = qc_cn_pipe(c, o, 1, s, S->sflags, o.algo == LDPC_ALGO_NOMS ? S->age : nullptr);
            if (e != LDPC_OK) return e;
            prof_end(slot_cn, s);
            const int slot_vn = prof_begin(1, s);
            e = qc_vn_refill(c, o, rf, s);
            if (e != LDPC_OK) return e;
            prof_end(slot_vn, s);
            count_launch(3);
            return LDPC_OK;
        }
        if (cw) {
            // wrong information bits of the frames retiring now, then the new frames' codewords
            e = enc_sim_errors(c, P, V, S->sflags, S->cwf, S->errs, s);
            if (e != LDPC_OK) return e;
            e = enc_sim_codewords(c, (int)slots, S->rlist, S->rcount, parity, S->fid, seed, S->cwf, s);
            if (e != LDPC_OK) return e;
        }
        const float qs = ldexpf(1.0f, o.frac_bits);
        if (i8 && cw)
            sim_channel_kernel<true, true><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N, parity,
                                                                   seed, fsig, s2, 1e30f, qs, S->cwf, NW);
        else if (i8)
            sim_channel_kernel<true, false><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N,
                                                                    parity, seed, fsig, s2, 1e30f, qs, nullptr, 0);
        else if (cw)
            sim_channel_kernel<false, true><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N,
                                                                    parity, seed, fsig, s2, o.clip, 1.0f, S->cwf, NW);
        else
            sim_channel_kernel<false, false><<<cblocks, 256, 0, s>>>(S->mu, S->rlist, S->rcount, S->fid, c->d.N,
                                                                     parity, seed, fsig, s2, o.clip, 1.0f, nullptr, 0);
        parity ^= 1;
        const int slot_cn = prof_begin(0, s);
        e = qc_cn_pipe(c, o, 1, s, S->sflags, o.algo == LDPC_ALGO_NOMS ? S->age : nullptr);
        if (e != LDPC_OK) return e;
        prof_end(slot_cn, s);
        const int slot_vn = prof_begin(1, s);
        e = qc_vn_refill(c, o, rf, s);
        if (e != LDPC_OK) return e;
        prof_end(slot_vn, s);
        count_launch(4);
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

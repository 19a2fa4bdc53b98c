// Decoding of general (not quasi-cyclic) LDPC codes: Algorithm 1 with the same
// pipelined check and variable passes as the QC decoder, their copy stages
// reading the edges of a row (consecutive, edges numbered row by row as in
// eq. simpleH) and of a variable (the column table) from index tables -- the
// role of the paper's LUT_c / LUT_v (Sec. IV-A) -- instead of circulant
// address arithmetic.  The first iteration starts from messages beta = mu
// written by an initialization pass; the syndrome for early stopping (tested after each complete iteration i >= 1)
// and the final ok flags gather the hard decisions through the row table.
#include "qc_device.cuh"

namespace ldpc {

// beta = mu on every edge of every package, in the form the check pass reads:
// sign(mu) phi(|mu|) for sum-product (scaled for FP16), the int8 word for min-sum.
// One thread per (package, edge, lane word).
template <int V, bool MS>
__global__ void sparse_init_kernel(const uint32_t *__restrict__ mu, uint32_t *__restrict__ msg, const int *__restrict__ col,
                                   int N, int E, int P) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)P * E * 32;
    if (i >= total) return;
    const int lane = (int)(i & 31);
    const long long pe = i >> 5;
    const int pk = (int)(pe / E), e = (int)(pe - (long long)pk * E);
    const int n = __ldg(col + e);
    if constexpr (MS) {
        msg[i] = mu[((size_t)pk * N + n) * 32 + lane];
    } else {
        const float *m = reinterpret_cast<const float *>(mu) + ((size_t)pk * N + n) * (32 * V) + lane * V;
        float b[V];
#pragma unroll
        for (int v = 0; v < V; ++v) b[v] = with_sign_of(phi_f(fabsf(m[v])) * XfScale<V>::store, m[v]);
        msg[i] = Lane<V>::pack(b);
    }
}

// syndrome of the hard decisions (eq. hrddcs) through the row table into flag word
// `word` (+v) of each package; one thread per row, a warp ORs its rows
template <int V>
__global__ void sparse_syndrome_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                       const uint32_t *__restrict__ hw, uint32_t *__restrict__ flags, int M, int N,
                                       int word) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int pk = blockIdx.y;
    uint32_t syn[V];
#pragma unroll
    for (int v = 0; v < V; ++v) syn[v] = 0u;
    if (m < M) {
        for (int e = __ldg(rp + m), e1 = __ldg(rp + m + 1); e < e1; ++e) {
            const uint32_t *h = hw + ((size_t)pk * N + __ldg(col + e)) * V;
#pragma unroll
            for (int v = 0; v < V; ++v) syn[v] ^= h[v];
        }
    }
    uint32_t *out = flags + (size_t)pk * 5 * V + word;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t any = __reduce_or_sync(0xffffffffu, syn[v]);
        if (any && (threadIdx.x & 31) == 0) atomicOr(out + v, any);
    }
}

static ldpc_status sparse_syndrome(ldpc_code c, int P, int V, int word, cudaStream_t s) {
    const dim3 grd((c->d.M + 255) / 256, P);
    if (V == 1) sparse_syndrome_kernel<1><<<grd, 256, 0, s>>>(c->sp.rp, c->sp.col, c->ws.hw, c->ws.flags, c->d.M, c->d.N, word);
    else if (V == 2) sparse_syndrome_kernel<2><<<grd, 256, 0, s>>>(c->sp.rp, c->sp.col, c->ws.hw, c->ws.flags, c->d.M, c->d.N, word);
    else sparse_syndrome_kernel<4><<<grd, 256, 0, s>>>(c->sp.rp, c->sp.col, c->ws.hw, c->ws.flags, c->d.M, c->d.N, word);
    count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status sparse_decode_device(ldpc_code c, int gamma, const ldpc_decode_opts &o, bool want_post, cudaStream_t s) {
    if (o.algo == LDPC_ALGO_NOMS) {
        set_error("the learned min-sum takes QC codes (parameters per circulant)");
        return LDPC_EUNSUPPORTED;
    }
    const int V = lanes_per_word(o.msg), W = 32 * V;
    const int P = (gamma + W - 1) / W;
    ldpc_status st = qc_init_flags(c, gamma, V, s);
    if (st != LDPC_OK) return st;
    LDPC_CUDA_TRY(cudaMemsetAsync(c->ws.hw, 0, (size_t)P * c->d.N * V * 4, s));
    st = qc_compact(c, P, V, s);  // every package starts active
    if (st != LDPC_OK) return st;
    {
        const long long n = (long long)P * c->d.E * 32;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        const uint32_t *mu = (const uint32_t *)c->ws.mu;
        uint32_t *msg = (uint32_t *)c->ws.msg;
        if (o.algo == LDPC_ALGO_MS) sparse_init_kernel<4, true><<<blocks, 256, 0, s>>>(mu, msg, c->sp.col, c->d.N, c->d.E, P);
        else if (V == 2) sparse_init_kernel<2, false><<<blocks, 256, 0, s>>>(mu, msg, c->sp.col, c->d.N, c->d.E, P);
        else sparse_init_kernel<1, false><<<blocks, 256, 0, s>>>(mu, msg, c->sp.col, c->d.N, c->d.E, P);
        count_launch(2);
        LDPC_CUDA_TRY(cudaGetLastError());
    }
    for (int it = 1; it <= o.max_iter; ++it) {
        const bool syn = o.early_stop && it >= 2;
        const int par = it & 1;
        if (syn) {  // early stop: the syndrome of the decisions after it - 1 complete iterations
            st = sparse_syndrome(c, P, V, (1 + par) * V, s);
            if (st != LDPC_OK) return st;
        }
        const int slot_cn = prof_begin(0, s);
        st = qc_cn_pipe_sparse(c, o, s);
        if (st != LDPC_OK) return st;
        prof_end(slot_cn, s);
        const int slot_vn = prof_begin(1, s);
        st = qc_vn_pipe_sparse(c, o, syn, want_post, it, par, s);
        if (st != LDPC_OK) return st;
        prof_end(slot_vn, s);
        count_launch(2);
        if (o.early_stop && it < o.max_iter) {
            st = qc_compact(c, P, V, s);
            if (st != LDPC_OK) return st;
            count_launch();
        }
    }
    st = sparse_syndrome(c, P, V, 4 * V, s);  // fin words: the last decisions
    if (st != LDPC_OK) return st;
    return qc_finish_frames(c, gamma, o, s);
}

}  // namespace ldpc

// api.cu -- the C ABI of include/wally.h: parameter set-up, the resident
// cluster store, and the batched evaluation pipeline (Alg. "Server
// Computation" of arXiv 2406.06761) built from the kernels in kernels.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>
#include <algorithm>
#include <thread>

#include "../../include/wally.h"
#include "host_nt.hpp"
#include "kernels.hpp"
#include "ctx_access.hpp"
#include "pir.hpp"
#include "plan.hpp"

using namespace wally;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) return fail(WALLY_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                          \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    cudaError_t ensure(size_t count)
    {
        if (count <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc((void **)&p, sizeof(T) * (count ? count : 1));
        if (e == cudaSuccess) n = count;
        else {
            p = nullptr;
            cudaGetLastError();  // a failed allocation must not surface at the next launch check
        }
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// Pinned host memory (asynchronous copies), grown on demand.
template <typename T>
struct PinnedBuf {
    T *p = nullptr;
    size_t n = 0;
    PinnedBuf() = default;
    PinnedBuf(const PinnedBuf &) = delete;
    PinnedBuf &operator=(const PinnedBuf &) = delete;
    ~PinnedBuf() { release(); }
    cudaError_t ensure(size_t count)
    {
        if (count <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost((void **)&p, sizeof(T) * (count ? count : 1));
        if (e == cudaSuccess) n = count;
        else {
            p = nullptr;
            cudaGetLastError();
        }
        return e;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

// Record e on st; inside a stream capture as an external event node, so that
// every replay of the graph writes the event's timestamp (read after the
// replay like any recorded event).
void record_event(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

// Per-launch CUDA events, summed per kernel kind when read.  Launches
// captured in a CUDA graph are timed by the graph's latest replay.
struct EventProfiler : Profiler {
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    cudaEvent_t open_[KK_COUNT] = {};
    cudaEvent_t take()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void begin(int kind, cudaStream_t st) override
    {
        open_[kind] = take();
        record_event(open_[kind], st);
    }
    void end(int kind, cudaStream_t st) override
    {
        cudaEvent_t e = take();
        record_event(e, st);
        recs.push_back({kind, open_[kind], e});
    }
    void reset()
    {
        used = 0;
        recs.clear();
    }
    // completion of every wave of the evaluation calls (their own event pool:
    // reading the kernel times does not recycle them)
    struct WaveRec {
        uint32_t call, queries;
        cudaEvent_t done;
    };
    std::vector<cudaEvent_t> wpool;
    size_t wused = 0;
    std::vector<cudaEvent_t> call_start;
    std::vector<WaveRec> waves;
    cudaEvent_t wtake()
    {
        if (wused == wpool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            wpool.push_back(e);
        }
        return wpool[wused++];
    }
    void call_begin(cudaStream_t st)
    {
        cudaEvent_t e = wtake();
        record_event(e, st);
        call_start.push_back(e);
    }
    void wave_end(cudaStream_t st, uint32_t queries)
    {
        if (call_start.empty()) return;
        cudaEvent_t e = wtake();
        record_event(e, st);
        waves.push_back({(uint32_t)call_start.size() - 1, queries, e});
    }
    void reset_waves()
    {
        wused = 0;
        call_start.clear();
        waves.clear();
    }
    ~EventProfiler()
    {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        for (cudaEvent_t e : wpool) cudaEventDestroy(e);
    }
};

// One independent evaluation workspace.  Lanes of a context share its
// read-only tables and cluster store, so waves on different lanes (different
// streams) may run concurrently.
struct Lane {
    uint32_t ws_wave = 0, ws_mmax = 0;
    DevBuf<u64> keysN, ctp, T, S, sc, dg, u, dd;
    DevBuf<u32> plan_u32;
    DevBuf<void *> plan_ptr;
    WavePlan wp{};
    // batch grouping
    DevBuf<u32> counts, cstart, fill, sorted_q;
    // compact cluster store: the chunks of the running wave, encoded, and
    // per cluster the cache index of its chunk 0
    DevBuf<u64> cache;
    DevBuf<u32> wchunk0, zlist;
    PinnedBuf<u32> h_counts, h_zlist;
    cudaEvent_t zlist_ev = nullptr;  // the last upload of h_zlist
    void release()
    {
        cache.release();
        wchunk0.release();
        zlist.release();
        h_counts.release();
        h_zlist.release();
        if (zlist_ev) cudaEventDestroy(zlist_ev);
        zlist_ev = nullptr;
        keysN.release();
        ctp.release();
        T.release();
        S.release();
        sc.release();
        dg.release();
        u.release();
        dd.release();
        plan_u32.release();
        plan_ptr.release();
        counts.release();
        cstart.release();
        fill.release();
        sorted_q.release();
        ws_wave = ws_mmax = 0;
    }
};

}  // namespace

struct wally_ctx {
    int device = 0;
    int num_sms = 0;
    uint32_t N = 0, log_n = 0, L = 0, d = 0, d_pad = 0, g = 0, h = 0;
    std::vector<uint64_t> mods;  // q_0..q_{L-1}, P, t
    uint64_t zeta_t = 0, k1 = 0, kg = 0, k1_inv = 0, kg_inv = 0;
    uint32_t drop0 = 0, drop1 = 0, bits0 = 0, bits1 = 0;  // response compression
    uint32_t max_wave = 1024;
    uint32_t store_req = WALLY_STORE_AUTO, store = WALLY_STORE_NTT, cache_chunks = 16;
    uint32_t lanes_pref = 2, ntt_cps = 0;  // launch shapes (wally_tuning)
    int smem_per_sm = 0, smem_reserved = 0;
    DevParams dp{};
    DevParams *d_dp = nullptr;
    std::vector<void *> tables;
    uint32_t *d_slot_pos = nullptr;
    uint32_t *d_err = nullptr;

    // cluster store
    uint32_t num_clusters = 0, m_max = 0, ts = 0;
    uint64_t total_chunks = 0;
    std::vector<uint32_t> h_chunks, h_chunk0;
    DevBuf<u64> ptxt;
    DevBuf<u32> d_chunks, d_chunk0;
    // compact store: the embeddings and their cluster index stay resident
    DevBuf<int8_t> emb;
    DevBuf<u64> row0;
    DevBuf<u32> csize, d_cc, d_ck;

    // evaluation workspaces
    Lane lanes[WALLY_MAX_LANES];
    // second stream of wally_eval_batch (waves alternate between lanes 0, 1)
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // host-buffer path staging
    DevBuf<u64> stage_ct[2], stage_key[2], stage_out[2];
    DevBuf<u32> stage_cluster[2];
    DevBuf<void *> stage_ptrs[2];
    PinnedBuf<u64> h_ct[2], h_out[2];
    PinnedBuf<u32> h_plan32[2];
    PinnedBuf<void *> h_planptr[2];
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
    // client and export temporaries
    DevBuf<u64> tmp;
    DevBuf<u32> tmp32;
    // index PIR: the table (NTT form, times 2^64), the monomials X^(-2^a),
    // and the expansion scratch
    uint32_t pir_rows = 0, pir_cols = 0, pir_levels = 0, pir_levels2 = 0;
    bool pir_derive = false;  // lower expansion keys derived by repeated substitution
    DevBuf<u64> pir_db, pir_mono, pir_E[2], pir_S, pir_keys, pir_out, pir_sc, pir_dg, pir_u, pir_dd;
    DevBuf<u32> pir_map;
    // MulPIR's second dimension: the extension basis (its own context for
    // the transforms), its constants on the device, and the buffers
    wally_ctx *ext = nullptr;
    DevBuf<ExtConst> ext_const;
    DevBuf<u64> pd_first, pd_col, pd_A, pd_B, pd_T, pd_X, pd_add, pd_out, pd_rlk;
    // optional per-launch timing
    bool prof_on = false;
    EventProfiler prof;
    Profiler *pr() { return prof_on ? &prof : nullptr; }

    size_t ctw() const { return (size_t)2 * L * N; }
    size_t chunk_words() const { return (size_t)L * N * d_pad; }
    bool compact() const { return store == WALLY_STORE_COMPACT; }
    size_t keysw() const { return (size_t)2 * L * 2 * (L + 1) * N; }
};

namespace {

int setup_tables(wally_ctx *c)
{
    const uint32_t M = c->L + 2;
    DevParams &dp = c->dp;
    memset(&dp, 0, sizeof(dp));
    dp.log_n = (int)c->log_n;
    dp.n = (int)c->N;
    dp.L = (int)c->L;
    dp.d = c->d;
    dp.d_pad = c->d_pad;
    dp.g = c->g;
    dp.h = c->h;
    for (uint32_t j = 0; j < M; j++) {
        const uint64_t p = c->mods[j];
        const uint64_t psi = (j == c->L + 1) ? c->zeta_t : root_2n(p, c->N);
        if (!psi) return fail(WALLY_EINVAL, "no 2N-th root of unity mod %llu", (unsigned long long)p);
        NttTables t = make_tables(p, psi, c->log_n);
        // interleaved (w, w') pairs, one 16-byte load per twiddle; and the
        // last radix-16 pass's entries 2^(S0+st) + (g << st | blk) again,
        // k-major (k = 2^st - 1 + blk, then group g), S0 = log2 N - 4
        const Tw *dptr[2], *lptr[2];
        const uint32_t G = c->N / 16, S0 = c->log_n - 4;
        for (int a = 0; a < 2; a++) {
            std::vector<uint64_t> pairs(2 * (size_t)c->N), last(2 * 15 * (size_t)G);
            for (uint32_t k = 0; k < c->N; k++) {
                pairs[2 * k] = a ? t.inv[k] : t.fwd[k];
                pairs[2 * k + 1] = a ? t.inv_s[k] : t.fwd_s[k];
            }
            for (uint32_t st = 0, k = 0; st < 4; st++)
                for (uint32_t blk = 0; blk < (1u << st); blk++, k++)
                    for (uint32_t g = 0; g < G; g++) {
                        const size_t src = ((size_t)1 << (S0 + st)) + (((size_t)g << st) | blk), dst = (size_t)k * G + g;
                        last[2 * dst] = pairs[2 * src];
                        last[2 * dst + 1] = pairs[2 * src + 1];
                    }
            void *ptr = nullptr, *lp = nullptr;
            CUDA_TRY(cudaMalloc(&ptr, 16 * (size_t)c->N));
            c->tables.push_back(ptr);
            CUDA_TRY(cudaMemcpy(ptr, pairs.data(), 16 * (size_t)c->N, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMalloc(&lp, 16 * 15 * (size_t)G));
            c->tables.push_back(lp);
            CUDA_TRY(cudaMemcpy(lp, last.data(), 16 * 15 * (size_t)G, cudaMemcpyHostToDevice));
            dptr[a] = (const Tw *)ptr;
            lptr[a] = (const Tw *)lp;
        }
        Mod &md = dp.m[j];
        md.p = p;
        md.two_p = 2 * p;
        md.four_p = 4 * p;
        md.np = (uint64_t)0 - p;
        md.mont_neg_inv = mont_neg_inv(p);
        const uint64_t r = (uint64_t)(((u128)1 << 64) % p);
        md.r2 = mulmod_h(r, r, p);
        md.n_inv = invmod_h(c->N % p, p);
        md.n_inv_s = shoup_of(md.n_inv, p);
        md.fwd = dptr[0];
        md.inv = dptr[1];
        md.fwd_last = lptr[0];
        md.inv_last = lptr[1];
    }
    // CRT constants.  Delta = floor(Q/t) by long division of the product.
    const uint64_t P = c->mods[c->L], t = c->mods[c->L + 1];
    std::vector<uint64_t> Q(1, 1);
    for (uint32_t i = 0; i < c->L; i++) Q = big_mul_small(Q, c->mods[i]);
    std::vector<uint64_t> delta = big_div_small(Q, t, nullptr);
    for (uint32_t j = 0; j < c->L; j++) {
        const uint64_t q = c->mods[j];
        dp.pinv[j] = invmod_h(P % q, q);
        dp.pinv_s[j] = shoup_of(dp.pinv[j], q);
        dp.pmodq[j] = P % q;
        dp.pmodq_s[j] = shoup_of(dp.pmodq[j], q);
        dp.delta[j] = big_mod_small(delta, q);
        dp.delta_s[j] = shoup_of(dp.delta[j], q);
        uint64_t qhat = 1;  // (Q/q_j) mod q_j
        for (uint32_t i = 0; i < c->L; i++)
            if (i != j) qhat = mulmod_h(qhat, c->mods[i] % q, q);
        dp.theta[j] = invmod_h(qhat, q);
        dp.theta_s[j] = shoup_of(dp.theta[j], q);
        for (uint32_t i = 0; i < c->L; i++) {
            dp.rs_inv[i][j] = i == j ? 0 : invmod_h(c->mods[i] % q, q);
            dp.rs_inv_s[i][j] = shoup_of(dp.rs_inv[i][j], q);
        }
    }
    // slot s = rho*N/2 + col is the evaluation at zeta^(+-3^col); the NTT
    // keeps the evaluation at zeta^(2 brv(i) + 1) in position i.
    std::vector<uint32_t> pos(c->N);
    const uint64_t two_n = 2 * (uint64_t)c->N;
    uint64_t e3 = 1;
    for (uint32_t col = 0; col < c->N / 2; col++) {
        for (uint32_t rho = 0; rho < 2; rho++) {
            const uint64_t e = rho ? two_n - e3 : e3;
            uint32_t nat = (uint32_t)((e - 1) / 2), r = 0;
            for (uint32_t b = 0; b < c->log_n; b++) r |= ((nat >> b) & 1u) << (c->log_n - 1 - b);
            pos[rho * (c->N / 2) + col] = r;
        }
        e3 = (e3 * 3) % two_n;
    }
    CUDA_TRY(cudaMalloc(&c->d_slot_pos, 4 * (size_t)c->N));
    CUDA_TRY(cudaMemcpy(c->d_slot_pos, pos.data(), 4 * (size_t)c->N, cudaMemcpyHostToDevice));
    dp.slot_pos = c->d_slot_pos;
    CUDA_TRY(cudaMalloc(&c->d_dp, sizeof(DevParams)));
    dp.self = c->d_dp;
    CUDA_TRY(cudaMemcpy(c->d_dp, &dp, sizeof(DevParams), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&c->d_err, 4));
    CUDA_TRY(cudaMemset(c->d_err, 0, 4));
    CUDA_TRY(set_kernel_attributes((int)c->log_n, c->g));
    return WALLY_OK;
}

uint64_t inv_mod_2n(uint64_t k, uint64_t two_n)
{
    for (uint64_t x = 1; x < two_n; x += 2)
        if ((k * x) % two_n == 1) return x;
    return 0;
}

// Wave workspace for W queries and up to W * m_max (query, chunk) pairs.
int ensure_workspace(wally_ctx *c, Lane &ln, uint32_t W, uint32_t m_max)
{
    if (ln.ws_wave >= W && ln.ws_mmax >= m_max && ln.keysN.p) return WALLY_OK;
    W = std::max(W, ln.ws_wave);
    m_max = std::max(m_max, std::max(ln.ws_mmax, 1u));
    const size_t ctw = c->ctw(), keysw = c->keysw(), N = c->N, L = c->L;
    const size_t pairs = (size_t)W * m_max;
    ln.keysN.release();
    ln.ctp.release();
    ln.T.release();
    ln.S.release();
    ln.sc.release();
    ln.dg.release();
    ln.u.release();
    ln.dd.release();
    const size_t items = std::max(pairs, (size_t)W);
    if (ln.keysN.ensure(W * keysw) != cudaSuccess || ln.ctp.ensure(W * (size_t)c->g * ctw) != cudaSuccess ||
        ln.T.ensure(pairs * c->h * ctw) != cudaSuccess || ln.S.ensure(items * ctw) != cudaSuccess ||
        ln.sc.ensure(items * ctw) != cudaSuccess || ln.dg.ensure(items * L * N) != cudaSuccess ||
        ln.u.ensure(items * 2 * (L + 1) * N) != cudaSuccess || ln.dd.ensure(items * (L + 1) * L * N) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the wave workspace (%u queries, %u chunks max)", W, m_max);
    // plan arrays: counts[4] | cluster[W] | pair_pos[P] | pair_k[P] | pair_off[W+1] | seg x3 [W]
    const size_t n32 = 4 + W + 2 * pairs + (W + 1) + 3 * (size_t)W;
    if (ln.plan_u32.ensure(n32) != cudaSuccess || ln.plan_ptr.ensure(3 * (size_t)W) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the wave plan");
    u32 *b = ln.plan_u32.p;
    WavePlan &wp = ln.wp;
    wp.counts = b;
    b += 4;
    wp.cluster = b;
    b += W;
    wp.pair_pos = b;
    b += pairs;
    wp.pair_k = b;
    b += pairs;
    wp.pair_off = b;
    b += W + 1;
    wp.seg_cluster = b;
    b += W;
    wp.seg_begin = b;
    b += W;
    wp.seg_end = b;
    void **pp = ln.plan_ptr.p;
    wp.src_ct = (const u64 **)pp;
    wp.src_key = (const u64 **)(pp + W);
    wp.dst_out = (u64 **)(pp + 2 * (size_t)W);
    ln.ws_wave = W;
    ln.ws_mmax = m_max;
    return WALLY_OK;
}

ClusterStore cluster_store(const wally_ctx *c)
{
    ClusterStore cs;
    cs.ptxt = c->ptxt.p;
    cs.chunk0 = c->d_chunk0.p;
    cs.chunks = c->d_chunks.p;
    cs.ts = c->ts;
    return cs;
}

RotArgs rot_args(Lane &ln)
{
    RotArgs a;
    memset(&a, 0, sizeof(a));
    a.sc = ln.sc.p;
    a.dg = ln.dg.p;
    a.u = ln.u.p;
    a.dd = ln.dd.p;
    return a;
}

// Steps a1-a5 for one wave whose plan inputs (counts[0], cluster, src_ct,
// src_key, dst_out of wp) are already on the device, in stream order.
int run_wave(wally_ctx *c, Lane &ln, const WavePlan &wp, uint32_t wave_len, const ClusterStore &cs, cudaStream_t st)
{
    const DevParams &dp = c->dp;
    const size_t ctw = c->ctw(), keysw = c->keysw();
    const uint32_t L = c->L, g = c->g, h = c->h;
    CUDA_TRY(launch_wave_plan(wp, c->d_chunks.p, wave_len, st, c->pr()));
    // a1: ciphertexts into slot 0 of the baby-step array, keys (Montgomery)
    CUDA_TRY(launch_to_ntt(dp, wp.src_ct, nullptr, 0, ln.ctp.p, (size_t)g * ctw, 2 * L, L, wave_len, wp.counts,
                           false, st, c->pr()));
    CUDA_TRY(launch_to_ntt(dp, wp.src_key, nullptr, 0, ln.keysN.p, keysw, 4 * L * (L + 1), L + 1, wave_len,
                           wp.counts, true, st, c->pr()));
    // a2: ct'[j] = Rot_1(ct'[j-1])
    for (uint32_t j = 1; j < g; j++) {
        RotArgs a = rot_args(ln);
        a.src = ln.ctp.p + (size_t)(j - 1) * ctw;
        a.src_stride = (size_t)g * ctw;
        a.dst = ln.ctp.p + (size_t)j * ctw;
        a.dst_stride = (size_t)g * ctw;
        a.key = ln.keysN.p;
        a.key_stride = keysw;
        a.n_max = wave_len;
        a.n_dev = wp.counts;
        a.galois = c->k1;
        a.prepared = j > 1;
        a.next_galois = j + 1 < g ? c->k1 : 0;
        CUDA_TRY(launch_rotate(dp, a, st, c->pr()));
    }
    // a3: T_i = sum_b P'_{k,i,b} ct'[b]
    CUDA_TRY(launch_mac(dp, cs, wp, ln.ctp.p, ln.T.p, wave_len, c->m_max, c->num_sms, st, c->pr()));
    // a4: S = T_{h-1}; S = Rot_g(S) + T_i, i = h-2 .. 0
    const uint32_t np_max = wave_len * c->m_max;
    for (int i = (int)h - 2; i >= 0; i--) {
        RotArgs a = rot_args(ln);
        if (i == (int)h - 2) {
            a.src = ln.T.p + (size_t)(h - 1) * ctw;
            a.src_stride = (size_t)h * ctw;
        } else {
            a.src = ln.S.p;
            a.src_stride = ctw;
        }
        a.dst = ln.S.p;
        a.dst_stride = ctw;
        a.add = ln.T.p + (size_t)i * ctw;
        a.add_stride = (size_t)h * ctw;
        a.key = ln.keysN.p + keysw / 2;
        a.key_stride = keysw;
        a.key_map = wp.pair_pos;
        a.n_max = np_max;
        a.n_dev = wp.counts + 1;
        a.galois = c->kg;
        a.prepared = i < (int)h - 2;
        a.next_galois = i > 0 ? c->kg : 0;
        CUDA_TRY(launch_rotate(dp, a, st, c->pr()));
    }
    // a5: back to coefficient form, into the caller's output
    if (h == 1) CUDA_TRY(launch_output(dp, wp, ln.T.p, ctw, np_max, st, c->pr()));
    else CUDA_TRY(launch_output(dp, wp, ln.S.p, ctw, np_max, st, c->pr()));
    return WALLY_OK;
}

// ---------------------------------------------------------------- compact cluster store
// Copy the chunk lists to the device (ln.zlist: [2][total], clusters then
// chunk indices) through the lane's pinned buffer, on `st`.
int upload_chunk_list(Lane &ln, const std::vector<uint32_t> &zc, const std::vector<uint32_t> &zk, cudaStream_t st)
{
    const size_t tot = zc.size();
    if (!ln.zlist_ev) CUDA_TRY(cudaEventCreateWithFlags(&ln.zlist_ev, cudaEventDisableTiming));
    else CUDA_TRY(cudaEventSynchronize(ln.zlist_ev));  // the previous upload has read h_zlist
    if (ln.h_zlist.ensure(2 * tot) != cudaSuccess || ln.zlist.ensure(2 * tot) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the chunk list");
    if (!tot) return WALLY_OK;
    memcpy(ln.h_zlist.p, zc.data(), 4 * tot);
    memcpy(ln.h_zlist.p + tot, zk.data(), 4 * tot);
    CUDA_TRY(cudaMemcpyAsync(ln.zlist.p, ln.h_zlist.p, 8 * tot, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(ln.zlist_ev, st));
    return WALLY_OK;
}

int ensure_cache(wally_ctx *c, Lane &ln)
{
    if (ln.cache.ensure((size_t)c->cache_chunks * c->chunk_words()) != cudaSuccess ||
        ln.wchunk0.ensure(std::max<uint32_t>(1, c->num_clusters)) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the chunk cache (%u chunks, %.2f GB)", c->cache_chunks,
                    c->cache_chunks * (double)c->chunk_words() * 8 / 1e9);
    return WALLY_OK;
}

// The cluster store a wave's multiply-accumulate reads: the resident NTT
// store, or the lane's cache after encode_wave.
ClusterStore wave_store(const wally_ctx *c, const Lane &ln)
{
    if (!c->compact()) return cluster_store(c);
    ClusterStore cs;
    cs.ptxt = ln.cache.p;
    cs.chunk0 = ln.wchunk0.p;
    cs.chunks = c->d_chunks.p;
    cs.ts = c->ts;
    return cs;
}

// Encode the wave's chunks (Alg. "Server Initialization", the same kernel as
// the NTT store) into the lane's cache; zlist: the call's uploaded chunk list.
int encode_wave(wally_ctx *c, Lane &ln, const Wave &w, const uint32_t *zlist, size_t total, cudaStream_t st)
{
    EncodeArgs a;
    memset(&a, 0, sizeof(a));
    a.emb = c->emb.p;
    a.row0 = c->row0.p;
    a.size = c->csize.p;
    a.chunk_cluster = zlist + w.z_off;
    a.chunk_k = zlist + total + w.z_off;
    a.total_chunks = w.nz;
    a.ptxt = ln.cache.p;
    a.ts = c->ts;
    a.chunk0_out = ln.wchunk0.p;
    CUDA_TRY(launch_encode_clusters(c->dp, a, st, c->pr()));
    return WALLY_OK;
}

// Device-resident batch over nl lanes (1 or 2): group by cluster on lanes[0]
// (on streams[0]), form the waves, and run them alternately on the lanes;
// with two lanes the second stream forks from and joins back into the first.
int eval_device(wally_ctx *c, Lane *const *lanes, const cudaStream_t *streams, int nl, uint32_t n, const uint32_t *ids,
                const uint64_t *cts, const uint64_t *keys, const uint32_t *input_index, const uint64_t *out_offsets,
                uint64_t *out)
{
    const uint32_t W = c->max_wave, K = c->num_clusters;
    Lane &l0 = *lanes[0];
    cudaStream_t st = streams[0];
    for (int i = 0; i < nl; i++) {
        int rc = ensure_workspace(c, *lanes[i], W, c->m_max);
        if (rc == WALLY_OK && c->compact()) rc = ensure_cache(c, *lanes[i]);
        if (rc) return rc;
    }
    if (l0.counts.ensure(K) != cudaSuccess || l0.cstart.ensure(K + 1) != cudaSuccess ||
        l0.fill.ensure(K) != cudaSuccess || l0.sorted_q.ensure(n) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the grouping arrays");
    if (c->prof_on) c->prof.call_begin(st);
    // a0: group by cluster (shared by the lanes)
    CUDA_TRY(launch_group(ids, n, K, l0.counts.p, l0.cstart.p, l0.fill.p, l0.sorted_q.p, c->d_err, st));
    std::vector<Wave> waves;
    std::vector<uint32_t> zc, zk;
    if (c->compact()) {
        if (l0.h_counts.ensure(K) != cudaSuccess) return fail(WALLY_ENOMEM, "cannot allocate the host counts");
        CUDA_TRY(cudaMemcpyAsync(l0.h_counts.p, l0.counts.p, 4 * (size_t)K, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        compact_waves(c->h_chunks.data(), c->num_clusters, c->cache_chunks, l0.h_counts.p, W, waves, zc, zk);
        int rc = upload_chunk_list(l0, zc, zk, st);
        if (rc) return rc;
    } else {
        fixed_waves(n, W, waves);
    }
    if (waves.size() < 2) nl = 1;
    if (nl > 1) {
        CUDA_TRY(cudaEventRecord(c->fork_ev, st));
        CUDA_TRY(cudaStreamWaitEvent(streams[1], c->fork_ev, 0));
    }
    for (size_t w = 0; w < waves.size(); w++) {
        Lane &ln = *lanes[w % nl];
        cudaStream_t s = streams[w % nl];
        const Wave &wv = waves[w];
        CUDA_TRY(launch_gather_wave(ln.wp, l0.sorted_q.p, ids, l0.cstart.p, K, wv.begin, wv.len, cts, keys,
                                    input_index, out_offsets, out, c->ctw(), c->keysw(), s));
        int rc = WALLY_OK;
        if (c->compact()) rc = encode_wave(c, ln, wv, l0.zlist.p, zc.size(), s);
        if (rc == WALLY_OK) rc = run_wave(c, ln, ln.wp, wv.len, wave_store(c, ln), s);
        if (rc) return rc;
        if (c->prof_on) c->prof.wave_end(s, wv.len);
    }
    if (nl > 1) {
        CUDA_TRY(cudaEventRecord(c->join_ev, streams[1]));
        CUDA_TRY(cudaStreamWaitEvent(st, c->join_ev, 0));
    }
    return WALLY_OK;
}

// ---------------------------------------------------------------- launch shapes
// Dynamic shared memory that holds the transform kernels to at most k CTAs
// per SM (0: what they need).
uint32_t ntt_smem_for(const wally_ctx *c, uint32_t k)
{
    const uint32_t need = (uint32_t)ntt_smem_need(c->log_n);
    if (!k || c->smem_per_sm <= 0) return 0;
    const int per = c->smem_per_sm / (int)(k + 1) - c->smem_reserved;  // k + 1 CTAs must not fit
    uint32_t dyn = per > 0 ? ((uint32_t)per + 15u) & ~15u : 0;
    if (dyn <= need) return 0;  // the need alone already limits the CTAs
    if (dyn > 225u * 1024u) return 0;  // the most the transform kernels are set up to take
    return dyn;
}

int apply_tuning(wally_ctx *c, const wally_tuning *t)
{
    if (!t->max_wave) return fail(WALLY_EINVAL, "max_wave must be positive");
    if (t->lanes != 1 && t->lanes != 2) return fail(WALLY_EINVAL, "lanes must be 1 or 2");
    if (t->mac_ctas_per_sm < 1 || t->mac_ctas_per_sm > 3) return fail(WALLY_EINVAL, "mac_ctas_per_sm must be 1..3");
    if (t->ks_core > 1) return fail(WALLY_EINVAL, "ks_core must be 0 or 1");
    if (t->mac_halves > 1) return fail(WALLY_EINVAL, "mac_halves must be 0 or 1");
    c->max_wave = t->max_wave;
    c->lanes_pref = t->lanes;
    c->dp.mac_ctas_per_sm = t->mac_ctas_per_sm;
    c->ntt_cps = t->ntt_ctas_per_sm;
    c->dp.ntt_smem = ntt_smem_for(c, t->ntt_ctas_per_sm);
    c->dp.ks_core = t->ks_core;
    c->dp.mac_halves = t->mac_halves;
    return WALLY_OK;
}

void current_tuning(const wally_ctx *c, wally_tuning *t)
{
    t->max_wave = c->max_wave;
    t->lanes = c->lanes_pref;
    t->mac_ctas_per_sm = c->dp.mac_ctas_per_sm ? c->dp.mac_ctas_per_sm : 3;
    t->ntt_ctas_per_sm = c->ntt_cps;
    t->ks_core = c->dp.ks_core;
    t->mac_halves = c->dp.mac_halves;
}

void release_waves(wally_ctx *c)
{
    for (Lane &ln : c->lanes) {
        ln.keysN.release();
        ln.ctp.release();
        ln.T.release();
        ln.S.release();
        ln.sc.release();
        ln.dg.release();
        ln.u.release();
        ln.dd.release();
        ln.plan_u32.release();
        ln.plan_ptr.release();
        ln.ws_wave = ln.ws_mmax = 0;
    }
}

// Oblivious expansion of nq queries over lv levels: pir_E[0] holds their
// NTT-form ciphertexts and pir_keys their keys (NTT form); on return
// pir_E[cur] holds [nq][2^lv] indicator ciphertexts.
// First expansion level whose key the client sends: 0, or with derived keys
// b = min(lv - 1, floor((log2 N - 1) / 2)), below which (N/2^a + 1)^2 =
// N/2^(a-1) + 1 (mod 2N) lets the key of level b serve every lower level.
uint32_t pir_key_base(const wally_ctx *c, uint32_t lv)
{
    if (!c->pir_derive || lv == 0) return 0;
    return std::min(lv - 1, (c->log_n - 1) / 2);
}

int pir_expand(wally_ctx *c, uint32_t nq, uint32_t lv, int &cur, cudaStream_t st)
{
    const size_t N = c->N, L = c->L, ctw = c->ctw(), keyw = c->keysw() / 2;
    const uint32_t b = pir_key_base(c, lv), nkeys = lv - b;
    cur = 0;
    for (uint32_t a = 0; a < lv; a++) {
        const u32 count = nq << a;
        CUDA_TRY(launch_pir_qmap(c->pir_map.p, count, a, st));
        RotArgs r;
        memset(&r, 0, sizeof(r));
        r.src = c->pir_E[cur].p;
        r.src_stride = ctw;
        r.dst = c->pir_S.p;
        r.dst_stride = ctw;
        r.key = c->pir_keys.p + (size_t)(a < b ? 0 : a - b) * keyw;
        r.key_stride = (size_t)nkeys * keyw;
        r.key_map = c->pir_map.p;
        r.n_max = count;
        r.galois = (uint64_t)(N >> (a < b ? b : a)) + 1;
        r.sc = c->pir_sc.p;
        r.dg = c->pir_dg.p;
        r.u = c->pir_u.p;
        r.dd = c->pir_dd.p;
        CUDA_TRY(launch_rotate(c->dp, r, st, c->pr()));
        // a level below b: the substitution of level b applied 2^(b - a) times
        for (uint32_t rep = 1; a < b && rep < (1u << (b - a)); rep++) {
            r.src = c->pir_S.p;
            CUDA_TRY(launch_rotate(c->dp, r, st, c->pr()));
        }
        CUDA_TRY(launch_pir_combine(c->dp, c->pir_E[cur].p, c->pir_S.p, c->pir_E[cur ^ 1].p,
                                    c->pir_mono.p + (size_t)a * L * N, count, a, st));
        cur ^= 1;
    }
    return WALLY_OK;
}

int pir_scratch(wally_ctx *c, uint32_t chunk, uint32_t lv, uint32_t cols)
{
    const size_t N = c->N, L = c->L, ctw = c->ctw(), keyw = c->keysw() / 2;
    const uint32_t full = 1u << lv, half = std::max(1u, full / 2);
    const size_t items = std::max<size_t>((size_t)chunk * half, chunk);
    if (c->pir_E[0].ensure((size_t)chunk * full * ctw) != cudaSuccess ||
        c->pir_E[1].ensure((size_t)chunk * full * ctw) != cudaSuccess || c->pir_S.ensure(items * ctw) != cudaSuccess ||
        c->pir_keys.ensure((size_t)chunk * std::max(lv, 1u) * keyw) != cudaSuccess ||
        c->pir_out.ensure((size_t)chunk * cols * ctw) != cudaSuccess || c->pir_sc.ensure(items * ctw) != cudaSuccess ||
        c->pir_dg.ensure(items * L * N) != cudaSuccess || c->pir_u.ensure(items * 2 * (L + 1) * N) != cudaSuccess ||
        c->pir_dd.ensure(items * (L + 1) * L * N) != cudaSuccess || c->pir_map.ensure(items) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the PIR scratch");
    return WALLY_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

namespace wally {
bool ctx_view(const wally_ctx *c, const DevParams **dp, int *device, uint32_t *n, uint32_t *L)
{
    if (!c) return false;
    *dp = &c->dp;
    *device = c->device;
    *n = c->N;
    *L = c->L;
    return true;
}

int ctx_fail(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace wally

extern "C" {

const char *wally_last_error(void) { return g_err.c_str(); }

int wally_setup_params(const wally_params *prm, wally_ctx **out)
{
    if (!prm || !out) return fail(WALLY_EINVAL, "null argument");
    *out = nullptr;
    if (prm->log_n < 12 || prm->log_n > 14) return fail(WALLY_EINVAL, "log_n must be 12, 13 or 14");
    if (prm->num_q < 1 || prm->num_q >= WALLY_MAX_LIMBS) return fail(WALLY_EINVAL, "num_q out of range");
    if (prm->q_bits < 20 || prm->q_bits > 61) return fail(WALLY_EINVAL, "q_bits out of range");
    if (prm->t_bits < 2 || prm->t_bits > 30) return fail(WALLY_EINVAL, "t_bits out of range");
    if (prm->dim < 1) return fail(WALLY_EINVAL, "dim must be positive");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || prm->device < 0 || prm->device >= ndev)
        return fail(WALLY_ECUDA, "CUDA device %d not available", prm->device);
    DeviceGuard guard(prm->device);
    wally_ctx *c = new wally_ctx();
    c->device = prm->device;
    c->log_n = prm->log_n;
    c->N = 1u << prm->log_n;
    c->L = prm->num_q;
    const uint64_t step = 2 * (uint64_t)c->N;
    uint64_t below = (uint64_t)1 << prm->q_bits;
    for (uint32_t i = 0; i < c->L; i++) {
        uint64_t q = prm->q ? prm->q[i] : prime_1mod_below(below, step);
        if (!q || !is_prime_u64(q) || q % step != 1) {
            delete c;
            return fail(WALLY_EINVAL, "no usable prime for limb %u", i);
        }
        c->mods.push_back(q);
        below = q;
    }
    uint64_t P = prm->p_special ? prm->p_special : prime_1mod_below(below, step);
    uint64_t t = prm->t ? prm->t : prime_1mod_below((uint64_t)1 << prm->t_bits, step);
    if (!P || !is_prime_u64(P) || P % step != 1 || !t || !is_prime_u64(t) || t % step != 1) {
        delete c;
        return fail(WALLY_EINVAL, "no usable special prime or plaintext modulus");
    }
    c->mods.push_back(P);
    c->mods.push_back(t);
    // the kernels feed residues of one modulus directly into transforms mod
    // another: every pair of ciphertext / special primes within a factor 2
    for (uint32_t a = 0; a <= c->L; a++)
        for (uint32_t b = 0; b <= c->L; b++)
            if (c->mods[a] >= 2 * c->mods[b]) {
                delete c;
                return fail(WALLY_EINVAL, "ciphertext and special primes must be within a factor of 2");
            }
    c->zeta_t = smallest_root_2n(t, c->N);
    c->d = prm->dim;
    uint32_t dp = 1, lg = 0;
    while (dp < prm->dim) { dp <<= 1; lg++; }
    c->d_pad = dp;
    c->g = 1u << ((lg + 1) / 2);
    if (prm->baby_steps) {
        const uint32_t g = prm->baby_steps;
        if (g < 2 || g > dp || (g & (g - 1))) {
            delete c;
            return fail(WALLY_EINVAL, "baby_steps = %u must be a power of two from 2 to d_pad = %u", g, dp);
        }
        c->g = g;
    }
    c->h = dp / c->g;
    if (c->d_pad > c->N / 2 || c->d_pad > 1024 || c->d_pad < 4) {
        delete c;
        return fail(WALLY_EINVAL, "dimension %u unsupported (d_pad must be 4..min(1024, N/2))", prm->dim);
    }
    c->k1 = 3;
    c->kg = powmod_h(3, c->g, step);
    c->k1_inv = inv_mod_2n(c->k1, step);
    c->kg_inv = inv_mod_2n(c->kg, step);
    c->max_wave = prm->max_wave ? prm->max_wave : 1024;
    if (prm->store > WALLY_STORE_COMPACT) {
        delete c;
        return fail(WALLY_EINVAL, "unknown cluster store %u", prm->store);
    }
    c->store_req = prm->store;
    c->store = prm->store == WALLY_STORE_COMPACT ? WALLY_STORE_COMPACT : WALLY_STORE_NTT;
    c->cache_chunks = prm->cache_chunks ? prm->cache_chunks : 16;
    {
        // response compression (Sec. 7): l0 = floor(log2(q'/t) - 2),
        // l1 = floor(log2(q'/t) - 2 - log2(z sqrt(2n/9))), z = 8
        const double r = std::log2((double)c->mods[c->L - 1] / (double)c->mods[c->L + 1]);
        const double l0 = std::floor(r - 2), l1 = std::floor(r - 2 - std::log2(8.0 * std::sqrt(2.0 * c->N / 9.0)));
        c->drop0 = l0 > 0 ? (uint32_t)l0 : 0;
        c->drop1 = l1 > 0 ? (uint32_t)l1 : 0;
        const uint64_t q = c->mods[c->L - 1];
        auto bits = [&](uint32_t l) {
            uint64_t mx = (q - 1 + (l ? (1ull << (l - 1)) : 0)) >> l;
            uint32_t b = 0;
            while (mx) { b++; mx >>= 1; }
            return b;
        };
        c->bits0 = bits(c->drop0);
        c->bits1 = bits(c->drop1);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
    cudaDeviceGetAttribute(&c->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device);
    int rc = setup_tables(c);
    if (rc != WALLY_OK) {
        std::string msg = g_err;
        wally_destroy(c);
        g_err = msg;
        return rc;
    }
    *out = c;
    return WALLY_OK;
}

void wally_destroy(wally_ctx *c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    for (void *p : c->tables) cudaFree(p);
    if (c->d_slot_pos) cudaFree(c->d_slot_pos);
    if (c->d_dp) cudaFree(c->d_dp);
    if (c->d_err) cudaFree(c->d_err);
    c->ptxt.release();
    c->d_chunks.release();
    c->d_chunk0.release();
    c->emb.release();
    c->row0.release();
    c->csize.release();
    c->d_cc.release();
    c->d_ck.release();
    for (Lane &ln : c->lanes) ln.release();
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    for (int b = 0; b < 2; b++) {
        c->stage_ct[b].release();
        c->stage_key[b].release();
        c->stage_out[b].release();
        c->stage_cluster[b].release();
        c->stage_ptrs[b].release();
        c->h_ct[b].release();
        c->h_out[b].release();
        c->h_plan32[b].release();
        c->h_planptr[b].release();
        if (c->in_done[b]) cudaEventDestroy(c->in_done[b]);
        if (c->comp_done[b]) cudaEventDestroy(c->comp_done[b]);
        if (c->out_done[b]) cudaEventDestroy(c->out_done[b]);
    }
    if (c->cin) cudaStreamDestroy(c->cin);
    if (c->cout) cudaStreamDestroy(c->cout);
    c->tmp.release();
    c->tmp32.release();
    for (DevBuf<u64> *b : {&c->pir_db, &c->pir_mono, &c->pir_E[0], &c->pir_E[1], &c->pir_S, &c->pir_keys, &c->pir_out,
                           &c->pir_sc, &c->pir_dg, &c->pir_u, &c->pir_dd, &c->pd_first, &c->pd_col, &c->pd_A, &c->pd_B,
                           &c->pd_T, &c->pd_X, &c->pd_add, &c->pd_out, &c->pd_rlk})
        b->release();
    c->pir_map.release();
    c->ext_const.release();
    if (c->ext) wally_destroy(c->ext);
    delete c;
}

int wally_query_info(const wally_ctx *c, wally_info *o)
{
    if (!c || !o) return fail(WALLY_EINVAL, "null argument");
    memset(o, 0, sizeof(*o));
    o->n = c->N;
    o->log_n = c->log_n;
    o->num_q = c->L;
    o->dim = c->d;
    o->d_pad = c->d_pad;
    o->g = c->g;
    o->h = c->h;
    o->num_clusters = c->num_clusters;
    for (uint32_t i = 0; i < c->L; i++) o->q[i] = c->mods[i];
    o->p_special = c->mods[c->L];
    o->t = c->mods[c->L + 1];
    o->zeta_t = c->zeta_t;
    o->k1 = c->k1;
    o->kg = c->kg;
    o->ct_words = c->ctw();
    o->keys_words = c->keysw();
    o->total_chunks = c->total_chunks;
    o->cluster_bytes = c->ptxt.n * 8;
    o->max_wave = c->max_wave;
    o->drop_c0 = c->drop0;
    o->drop_c1 = c->drop1;
    o->compressed_bytes = (uint64_t)(c->N / 8) * (c->bits0 + c->bits1);
    o->store = c->num_clusters ? c->store : c->store_req;
    o->cache_chunks = c->cache_chunks;
    if (c->compact()) o->cluster_bytes = c->emb.n;
    return WALLY_OK;
}

int wally_load_clusters(wally_ctx *c, uint32_t K, const uint32_t *sizes, const int8_t *emb, void *stream)
{
    if (!c || (K && !sizes)) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint32_t> chunks(K), chunk0(K);
    std::vector<uint64_t> row0(K);
    uint64_t rows = 0, Z = 0;
    uint32_t m_max = 1;
    for (uint32_t i = 0; i < K; i++) {
        uint32_t m = std::max<uint32_t>(1, (sizes[i] + c->N - 1) / c->N);
        if (m >= c->g)
            return fail(WALLY_EINVAL,
                        "cluster %u needs %u chunks; the diagonal split needs fewer than g = %u "
                        "(baby_steps = d_pad allows up to d_pad - 1)",
                        i, m, c->g);
        chunks[i] = m;
        chunk0[i] = (uint32_t)Z;
        row0[i] = rows;
        rows += sizes[i];
        Z += m;
        m_max = std::max(m_max, m);
    }
    if (rows && !emb) return fail(WALLY_EINVAL, "null embeddings");
    // tile width: one tile of d_pad * ts words is 64 KB of shared memory
    uint32_t ts = std::max<uint32_t>(1, 8192 / c->d_pad);
    ts = std::min<uint32_t>(ts, 64);
    const size_t words = (size_t)Z * c->chunk_words();
    c->ptxt.release();
    c->emb.release();
    c->row0.release();
    c->csize.release();
    c->d_cc.release();
    c->d_ck.release();
    c->num_clusters = 0;
    uint32_t store = c->store_req;
    if (store == WALLY_STORE_AUTO) {
        size_t free_b = 0, total_b = 0;
        CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        store = words * 8.0 <= 0.6 * (double)free_b ? WALLY_STORE_NTT : WALLY_STORE_COMPACT;
    }
    if (store == WALLY_STORE_COMPACT && c->cache_chunks < m_max)
        return fail(WALLY_EINVAL, "cache_chunks = %u is below the largest cluster's %u chunks", c->cache_chunks, m_max);
    if (store == WALLY_STORE_NTT && c->ptxt.ensure(words) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate %.1f GB for the encoded clusters", words * 8.0 / 1e9);
    std::vector<uint32_t> chunk_cluster(Z), chunk_k(Z);
    for (uint32_t i = 0; i < K; i++)
        for (uint32_t k = 0; k < chunks[i]; k++) {
            chunk_cluster[chunk0[i] + k] = i;
            chunk_k[chunk0[i] + k] = k;
        }
    if (c->emb.ensure(std::max<size_t>(1, rows * c->d)) != cudaSuccess ||
        c->row0.ensure(std::max<size_t>(1, K)) != cudaSuccess || c->csize.ensure(std::max<size_t>(1, K)) != cudaSuccess ||
        c->d_cc.ensure(std::max<size_t>(1, Z)) != cudaSuccess || c->d_ck.ensure(std::max<size_t>(1, Z)) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate %.2f GB for the embeddings", rows * (double)c->d / 1e9);
    if (rows) CUDA_TRY(cudaMemcpyAsync(c->emb.p, emb, rows * c->d, cudaMemcpyHostToDevice, st));
    if (K) {
        CUDA_TRY(cudaMemcpyAsync(c->row0.p, row0.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(c->csize.p, sizes, 4 * (size_t)K, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(c->d_cc.p, chunk_cluster.data(), 4 * (size_t)Z, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(c->d_ck.p, chunk_k.data(), 4 * (size_t)Z, cudaMemcpyHostToDevice, st));
    }
    c->ts = ts;
    if (store == WALLY_STORE_NTT) {
        for (uint64_t z0 = 0; z0 < Z; z0 += 65535) {
            EncodeArgs a;
            memset(&a, 0, sizeof(a));
            a.emb = c->emb.p;
            a.row0 = c->row0.p;
            a.size = c->csize.p;
            a.chunk_cluster = c->d_cc.p + z0;
            a.chunk_k = c->d_ck.p + z0;
            a.total_chunks = (uint32_t)std::min<uint64_t>(65535, Z - z0);
            a.ptxt = c->ptxt.p + z0 * c->chunk_words();
            a.ts = ts;
            CUDA_TRY(launch_encode_clusters(c->dp, a, st));
        }
    }
    if (c->d_chunks.ensure(std::max<uint32_t>(K, 1)) != cudaSuccess ||
        c->d_chunk0.ensure(std::max<uint32_t>(K, 1)) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the cluster index");
    CUDA_TRY(cudaMemcpyAsync(c->d_chunks.p, chunks.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(c->d_chunk0.p, chunk0.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (store == WALLY_STORE_NTT) {
        // the encoded store replaces the embeddings
        c->emb.release();
        c->row0.release();
        c->csize.release();
        c->d_cc.release();
        c->d_ck.release();
    }
    for (Lane &ln : c->lanes) {
        // a previous store's per-wave cache no longer matches
        ln.cache.release();
        ln.wchunk0.release();
    }
    c->store = store;
    c->num_clusters = K;
    c->m_max = m_max;
    c->total_chunks = Z;
    c->h_chunks = chunks;
    c->h_chunk0 = chunk0;
    return WALLY_OK;
}

int wally_cluster_chunks(const wally_ctx *c, uint32_t id, uint32_t *m_out)
{
    if (!c || !m_out) return fail(WALLY_EINVAL, "null argument");
    if (id >= c->num_clusters) return fail(WALLY_EINVAL, "cluster id %u out of range (%u clusters)", id, c->num_clusters);
    *m_out = c->h_chunks[id];
    return WALLY_OK;
}

int wally_export_cluster(wally_ctx *c, uint32_t id, uint64_t *out, void *stream)
{
    if (!c || !out) return fail(WALLY_EINVAL, "null argument");
    if (id >= c->num_clusters) return fail(WALLY_EINVAL, "cluster id %u out of range", id);
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->compact()) {
        CUDA_TRY(launch_export_cluster(c->dp, cluster_store(c), id, c->h_chunks[id], out, st));
        return WALLY_OK;
    }
    // compact store: encode the cluster's chunks into scratch, then export
    const uint32_t m = c->h_chunks[id];
    if (c->tmp.ensure((size_t)m * c->chunk_words()) != cudaSuccess || c->tmp32.ensure(c->num_clusters) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the export scratch");
    EncodeArgs a;
    memset(&a, 0, sizeof(a));
    a.emb = c->emb.p;
    a.row0 = c->row0.p;
    a.size = c->csize.p;
    a.chunk_cluster = c->d_cc.p + c->h_chunk0[id];
    a.chunk_k = c->d_ck.p + c->h_chunk0[id];
    a.total_chunks = m;
    a.ptxt = c->tmp.p;
    a.ts = c->ts;
    a.chunk0_out = c->tmp32.p;
    CUDA_TRY(launch_encode_clusters(c->dp, a, st));
    ClusterStore cs;
    cs.ptxt = c->tmp.p;
    cs.chunk0 = c->tmp32.p;
    cs.chunks = c->d_chunks.p;
    cs.ts = c->ts;
    CUDA_TRY(launch_export_cluster(c->dp, cs, id, m, out, st));
    return WALLY_OK;
}

int wally_eval_batch_lane(wally_ctx *c, uint32_t lane, uint32_t n, const uint32_t *ids, const uint64_t *cts,
                          const uint64_t *keys, const uint32_t *input_index, const uint64_t *out_offsets, uint64_t *out,
                          void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (!c->num_clusters) return fail(WALLY_ESTATE, "no clusters loaded");
    if (n == 0) return WALLY_OK;
    if (!ids || !cts || !keys || !out_offsets || !out) return fail(WALLY_EINVAL, "null argument");
    if (!aligned16(cts) || !aligned16(keys) || !aligned16(out)) return fail(WALLY_EINVAL, "buffers must be 16-byte aligned");
    if (lane >= WALLY_MAX_LANES) return fail(WALLY_EINVAL, "lane %u out of range (%d lanes)", lane, WALLY_MAX_LANES);
    DeviceGuard guard(c->device);
    Lane *ls[1] = {&c->lanes[lane]};
    cudaStream_t ss[1] = {(cudaStream_t)stream};
    return eval_device(c, ls, ss, 1, n, ids, cts, keys, input_index, out_offsets, out);
}

// Waves alternate between lane 0 on the caller's stream and lane 1 on the
// context's second stream (forked from and joined back into the caller's
// stream with events), so that one wave's kernels fill the tails and the
// memory-bound phases of the other's.
int wally_eval_batch(wally_ctx *c, uint32_t n, const uint32_t *ids, const uint64_t *cts, const uint64_t *keys,
                     const uint32_t *input_index, const uint64_t *out_offsets, uint64_t *out, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if ((n <= c->max_wave || c->lanes_pref == 1) && !c->compact())
        return wally_eval_batch_lane(c, 0, n, ids, cts, keys, input_index, out_offsets, out, stream);
    if (!c->num_clusters) return fail(WALLY_ESTATE, "no clusters loaded");
    if (n == 0) return WALLY_OK;
    if (!ids || !cts || !keys || !out_offsets || !out) return fail(WALLY_EINVAL, "null argument");
    if (!aligned16(cts) || !aligned16(keys) || !aligned16(out)) return fail(WALLY_EINVAL, "buffers must be 16-byte aligned");
    DeviceGuard guard(c->device);
    if (!c->side) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    Lane *ls[2] = {&c->lanes[0], &c->lanes[1]};
    cudaStream_t ss[2] = {(cudaStream_t)stream, c->side};
    return eval_device(c, ls, ss, (int)c->lanes_pref, n, ids, cts, keys, input_index, out_offsets, out);
}

// Copy many host blocks (dst, src, bytes) with a few threads: the small
// per-query ciphertexts and outputs of the host path are gathered into and
// scattered from one contiguous pinned buffer a wave, so that each crosses
// to the device in one large transfer instead of hundreds of small ones.
struct HostCopy {
    void *dst;
    const void *src;
    size_t bytes;
};

void parallel_copy(const std::vector<HostCopy> &jobs)
{
    const size_t n = jobs.size();
    if (!n) return;
    unsigned hw = std::thread::hardware_concurrency();
    const size_t nt = std::min<size_t>(std::max(1u, std::min(hw, 16u)), (n + 15) / 16);
    auto work = [&](size_t t) {
        for (size_t i = t; i < n; i += nt) memcpy(jobs[i].dst, jobs[i].src, jobs[i].bytes);
    };
    if (nt <= 1) {
        work(0);
        return;
    }
    std::vector<std::thread> th;
    for (size_t t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (std::thread &x : th) x.join();
}

int wally_eval_batch_host(wally_ctx *c, uint32_t n, const uint32_t *ids, const uint64_t *cts, const uint64_t *keys,
                          const uint32_t *input_index, const uint64_t *out_offsets, uint64_t *out, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (!c->num_clusters) return fail(WALLY_ESTATE, "no clusters loaded");
    if (n == 0) return WALLY_OK;
    if (!ids || !cts || !keys || !out_offsets || !out) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t K = c->num_clusters, W = c->max_wave;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= K) return fail(WALLY_EINVAL, "query %u names cluster %u of %u", q, ids[q], K);
    Lane &ln = c->lanes[0];
    int rc = ensure_workspace(c, ln, W, c->m_max);
    if (rc == WALLY_OK && c->compact()) rc = ensure_cache(c, ln);
    if (rc) return rc;
    const size_t ctw = c->ctw(), keysw = c->keysw();
    for (int b = 0; b < 2; b++) {
        if (c->stage_ct[b].ensure((size_t)W * ctw) != cudaSuccess ||
            c->stage_key[b].ensure((size_t)W * keysw) != cudaSuccess ||
            c->stage_out[b].ensure((size_t)W * c->m_max * ctw) != cudaSuccess ||
            c->stage_cluster[b].ensure(W + 4) != cudaSuccess || c->stage_ptrs[b].ensure(3 * (size_t)W) != cudaSuccess ||
            c->h_ct[b].ensure((size_t)W * ctw) != cudaSuccess ||
            c->h_out[b].ensure((size_t)W * c->m_max * ctw) != cudaSuccess ||
            c->h_plan32[b].ensure((size_t)W + 4) != cudaSuccess || c->h_planptr[b].ensure(3 * (size_t)W) != cudaSuccess)
            return fail(WALLY_ENOMEM, "cannot allocate the staging buffers");
    }
    // host-side grouping by cluster (counting sort; stable)
    std::vector<uint32_t> start(K + 1, 0), order(n);
    for (uint32_t q = 0; q < n; q++) start[ids[q] + 1]++;
    for (uint32_t k = 0; k < K; k++) start[k + 1] += start[k];
    {
        std::vector<uint32_t> fillh(start.begin(), start.end() - 1);
        for (uint32_t q = 0; q < n; q++) order[fillh[ids[q]]++] = q;
    }
    std::vector<Wave> waves;
    std::vector<uint32_t> zc, zk;
    if (c->compact()) {
        std::vector<uint32_t> cnt(K);
        for (uint32_t k = 0; k < K; k++) cnt[k] = start[k + 1] - start[k];
        compact_waves(c->h_chunks.data(), c->num_clusters, c->cache_chunks, cnt.data(), W, waves, zc, zk);
        rc = upload_chunk_list(ln, zc, zk, st);
        if (rc) return rc;
    } else {
        fixed_waves(n, W, waves);
    }
    if (!c->cin) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->cin, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamCreateWithFlags(&c->cout, cudaStreamNonBlocking));
        for (int b = 0; b < 2; b++) {
            CUDA_TRY(cudaEventCreateWithFlags(&c->in_done[b], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&c->comp_done[b], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&c->out_done[b], cudaEventDisableTiming));
        }
    }
    cudaStream_t cin = c->cin, cout_ = c->cout;
    for (int b = 0; b < 2; b++) {
        CUDA_TRY(cudaEventRecord(c->in_done[b], st));
        CUDA_TRY(cudaEventRecord(c->comp_done[b], st));
        CUDA_TRY(cudaEventRecord(c->out_done[b], st));
    }
    // per buffer: the wave it holds and its (query, chunk) offsets
    std::vector<uint32_t> pair_off[2] = {std::vector<uint32_t>(W + 1), std::vector<uint32_t>(W + 1)};
    int held[2] = {-1, -1};
    std::vector<HostCopy> jobs;
    jobs.reserve(W);
    // outputs of wave w (in buffer w & 1), already read back: to the caller
    auto scatter = [&](int w) -> int {
        const int b = w & 1;
        if (cudaEventSynchronize(c->out_done[b]) != cudaSuccess) return fail(WALLY_ECUDA, "output read-back failed");
        const Wave &wv = waves[w];
        jobs.clear();
        for (uint32_t i = 0; i < wv.len; i++) {
            const uint32_t q = order[wv.begin + i];
            const uint32_t m = c->h_chunks[ids[q]];
            jobs.push_back({out + out_offsets[q] * ctw, c->h_out[b].p + (size_t)pair_off[b][i] * ctw, 8 * ctw * m});
        }
        parallel_copy(jobs);
        held[b] = -1;
        return WALLY_OK;
    };
    rc = WALLY_OK;
    for (size_t wave = 0; wave < waves.size() && rc == WALLY_OK; wave++) {
        const int b = wave & 1;
        const uint32_t wb = waves[wave].begin, len = waves[wave].len;
        // the pinned buffers of b are free once the uploads of wave - 2 are
        // done and its outputs have been handed over
        if (held[b] >= 0 && (rc = scatter(held[b])) != WALLY_OK) break;
        if (cudaEventSynchronize(c->in_done[b]) != cudaSuccess) {
            rc = fail(WALLY_ECUDA, "input upload failed");
            break;
        }
        uint32_t *p32 = c->h_plan32[b].p;
        void **pp = c->h_planptr[b].p;
        std::vector<uint32_t> &po = pair_off[b];
        p32[0] = len;
        p32[1] = p32[2] = p32[3] = 0;
        po[0] = 0;
        jobs.clear();
        for (uint32_t i = 0; i < len; i++) {
            const uint32_t q = order[wb + i];
            const uint32_t src = input_index ? input_index[q] : q;
            p32[4 + i] = ids[q];
            po[i + 1] = po[i] + c->h_chunks[ids[q]];
            pp[i] = c->stage_ct[b].p + (size_t)i * ctw;
            pp[W + i] = c->stage_key[b].p + (size_t)i * keysw;
            pp[2 * (size_t)W + i] = c->stage_out[b].p + (size_t)po[i] * ctw;
            jobs.push_back({c->h_ct[b].p + (size_t)i * ctw, cts + (size_t)src * ctw, 8 * ctw});
        }
        parallel_copy(jobs);
        // uploads wait until the compute of wave - 2 has read the device buffers
        CUDA_TRY(cudaStreamWaitEvent(cin, c->comp_done[b], 0));
        CUDA_TRY(cudaMemcpyAsync(c->stage_ct[b].p, c->h_ct[b].p, 8 * ctw * len, cudaMemcpyHostToDevice, cin));
        for (uint32_t i = 0; i < len; i++) {
            const uint32_t q = order[wb + i];
            const uint32_t src = input_index ? input_index[q] : q;
            CUDA_TRY(cudaMemcpyAsync(c->stage_key[b].p + (size_t)i * keysw, keys + (size_t)src * keysw, 8 * keysw,
                                     cudaMemcpyHostToDevice, cin));
        }
        WavePlan wp = ln.wp;
        wp.counts = c->stage_cluster[b].p;
        wp.cluster = c->stage_cluster[b].p + 4;
        wp.src_ct = (const u64 **)c->stage_ptrs[b].p;
        wp.src_key = (const u64 **)(c->stage_ptrs[b].p + W);
        wp.dst_out = (u64 **)(c->stage_ptrs[b].p + 2 * (size_t)W);
        CUDA_TRY(cudaMemcpyAsync(wp.counts, p32, 4 * ((size_t)len + 4), cudaMemcpyHostToDevice, cin));
        CUDA_TRY(cudaMemcpyAsync(c->stage_ptrs[b].p, pp, sizeof(void *) * 3 * (size_t)W, cudaMemcpyHostToDevice, cin));
        CUDA_TRY(cudaEventRecord(c->in_done[b], cin));
        CUDA_TRY(cudaStreamWaitEvent(st, c->in_done[b], 0));
        CUDA_TRY(cudaStreamWaitEvent(st, c->out_done[b], 0));
        if (c->compact()) rc = encode_wave(c, ln, waves[wave], ln.zlist.p, zc.size(), st);
        if (rc == WALLY_OK) rc = run_wave(c, ln, wp, len, wave_store(c, ln), st);
        if (rc) break;
        if (c->prof_on) c->prof.wave_end(st, len);
        CUDA_TRY(cudaEventRecord(c->comp_done[b], st));
        CUDA_TRY(cudaStreamWaitEvent(cout_, c->comp_done[b], 0));
        CUDA_TRY(cudaMemcpyAsync(c->h_out[b].p, c->stage_out[b].p, 8 * ctw * po[len], cudaMemcpyDeviceToHost, cout_));
        CUDA_TRY(cudaEventRecord(c->out_done[b], cout_));
        held[b] = (int)wave;
    }
    for (int k = 0; k < 2 && rc == WALLY_OK; k++) {
        const int b = (int)((waves.size() + k) & 1);  // the older wave first
        if (held[b] >= 0) rc = scatter(held[b]);
    }
    cudaStreamSynchronize(cin);
    cudaStreamSynchronize(cout_);
    cudaStreamSynchronize(st);
    return rc;
}

int wally_rotate(wally_ctx *c, uint32_t n, uint64_t k, const uint64_t *cts, const uint64_t *keys, uint64_t *out,
                 void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!cts || !keys || !out) return fail(WALLY_EINVAL, "null argument");
    if ((k & 1) == 0 || k >= 2 * (uint64_t)c->N) return fail(WALLY_EINVAL, "Galois element must be odd and < 2N");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    Lane &ln = c->lanes[0];
    int rc = ensure_workspace(c, ln, c->max_wave, std::max<uint32_t>(c->m_max, 1));
    if (rc) return rc;
    const size_t ctw = c->ctw(), keyw = c->keysw() / 2;
    const uint32_t chunk = c->max_wave;
    for (uint32_t x0 = 0; x0 < n; x0 += chunk) {
        const uint32_t cnt = std::min(chunk, n - x0);
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, cts + (size_t)x0 * ctw, ctw, ln.S.p, ctw, 2 * c->L, c->L, cnt, nullptr,
                               false, st));
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, keys + (size_t)x0 * keyw, keyw, ln.keysN.p, keyw,
                               2 * c->L * (c->L + 1), c->L + 1, cnt, nullptr, true, st));
        RotArgs a = rot_args(ln);
        a.src = ln.S.p;
        a.src_stride = ctw;
        a.dst = ln.S.p;
        a.dst_stride = ctw;
        a.key = ln.keysN.p;
        a.key_stride = keyw;
        a.n_max = cnt;
        a.galois = k;
        CUDA_TRY(launch_rotate(c->dp, a, st));
        CUDA_TRY(launch_from_ntt(c->dp, ln.S.p, out + (size_t)x0 * ctw, 2 * c->L, c->L, cnt, st));
    }
    return WALLY_OK;
}

int wally_get_tuning(const wally_ctx *c, wally_tuning *out)
{
    if (!c || !out) return fail(WALLY_EINVAL, "null argument");
    current_tuning(c, out);
    return WALLY_OK;
}

int wally_set_tuning(wally_ctx *c, const wally_tuning *t)
{
    if (!c || !t) return fail(WALLY_EINVAL, "null argument");
    return apply_tuning(c, t);
}

// Mean device milliseconds per query of the sample under shape t (one
// untimed call, then reps timed ones), or -1 if its workspace does not fit.
int time_shape(wally_ctx *c, const wally_tuning &t, uint32_t reps, uint32_t n, const uint32_t *ids,
               const uint64_t *cts, const uint64_t *keys, const uint32_t *input_index, const uint64_t *out_offsets,
               uint64_t *out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *ms_out)
{
    release_waves(c);
    int rc = apply_tuning(c, &t);
    if (rc) return rc;
    rc = wally_eval_batch(c, n, ids, cts, keys, input_index, out_offsets, out, st);
    if (rc == WALLY_ENOMEM) {
        *ms_out = -1;
        return WALLY_OK;
    }
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(e0, st));
    for (uint32_t k = 0; k < reps; k++) {
        rc = wally_eval_batch(c, n, ids, cts, keys, input_index, out_offsets, out, st);
        if (rc) return rc;
    }
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *ms_out = (double)ms / reps / n;
    return WALLY_OK;
}

int wally_autotune(wally_ctx *c, const wally_tuning *cand, uint32_t nc, uint32_t reps, uint32_t n, const uint32_t *ids,
                   const uint64_t *cts, const uint64_t *keys, const uint32_t *input_index, const uint64_t *out_offsets,
                   uint64_t *out, wally_tuning *tried, double *ms_per_query, uint32_t *num_tried, uint32_t *best,
                   void *stream)
{
    if (!c || !best) return fail(WALLY_EINVAL, "null argument");
    if (!c->num_clusters) return fail(WALLY_ESTATE, "no clusters loaded");
    if (!n) return fail(WALLY_EINVAL, "empty sample");
    if (!cand && nc) return fail(WALLY_EINVAL, "num_candidates must be 0 without candidates");
    if (cand && !nc) return fail(WALLY_EINVAL, "no candidates");
    for (uint32_t i = 0; cand && i < nc; i++)
        if (!cand[i].max_wave || (cand[i].lanes != 1 && cand[i].lanes != 2) || cand[i].mac_ctas_per_sm < 1 ||
            cand[i].mac_ctas_per_sm > 3 || cand[i].ks_core > 1 || cand[i].mac_halves > 1)
            return fail(WALLY_EINVAL, "invalid candidate shape %u", i);
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    wally_tuning keep;
    current_tuning(c, &keep);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    reps = std::max(reps, 1u);
    std::vector<wally_tuning> done;
    std::vector<double> ms;
    int rc = WALLY_OK;
    auto run = [&](const wally_tuning &t) {
        double m = -1;
        if (rc == WALLY_OK) rc = time_shape(c, t, reps, n, ids, cts, keys, input_index, out_offsets, out, st, e0, e1, &m);
        done.push_back(t);
        ms.push_back(m);
    };
    auto best_of = [&]() {
        int bi = -1;
        for (size_t i = 0; i < ms.size(); i++)
            if (ms[i] > 0 && (bi < 0 || ms[i] < ms[bi])) bi = (int)i;
        return bi;
    };
    if (cand) {
        for (uint32_t i = 0; i < nc && rc == WALLY_OK; i++) run(cand[i]);
    } else {
        for (uint32_t w : {512u, 1024u, 2048u})
            for (uint32_t l : {1u, 2u}) run(wally_tuning{w, l, 3, 0, 0, 0});
        const int b1 = best_of();
        if (rc == WALLY_OK && b1 >= 0) {
            const wally_tuning base = done[b1];
            for (uint32_t m : {2u, 3u})
                for (uint32_t k : {0u, 2u})
                    if (!(m == 3 && k == 0)) run(wally_tuning{base.max_wave, base.lanes, m, k, 0, 0});
        }
        const int b2 = best_of();
        if (rc == WALLY_OK && b2 >= 0) {
            wally_tuning t = done[b2];
            t.ks_core = 1;
            run(t);
        }
        const int b3 = best_of();
        if (rc == WALLY_OK && b3 >= 0) {
            wally_tuning t = done[b3];
            t.mac_halves = 1;
            run(t);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release_waves(c);
    const int bi = best_of();
    if (rc == WALLY_OK && bi < 0) rc = fail(WALLY_ENOMEM, "no candidate shape fits in device memory");
    if (rc) {
        apply_tuning(c, &keep);
        return rc;
    }
    const size_t cap = cand ? nc : WALLY_AUTOTUNE_MAX;
    for (size_t i = 0; i < done.size() && i < cap; i++) {
        if (tried) tried[i] = done[i];
        if (ms_per_query) ms_per_query[i] = ms[i];
    }
    if (num_tried) *num_tried = (uint32_t)done.size();
    *best = (uint32_t)bi;
    return apply_tuning(c, &done[bi]);
}

// ---------------------------------------------------------------- index PIR (Sec. 4.2)
int wally_pir_load(wally_ctx *c, uint32_t rows, uint32_t cols, const uint64_t *table, void *stream)
{
    if (!c || !table) return fail(WALLY_EINVAL, "null argument");
    if (rows < 1 || rows > 4096 || cols < 1) return fail(WALLY_EINVAL, "table of %u x %u (rows 1..4096)", rows, cols);
    if ((uint64_t)cols * c->L > 65535) return fail(WALLY_EINVAL, "too many columns");
    const uint64_t t = c->mods[c->L + 1];
    const size_t N = c->N, L = c->L, P = (size_t)rows * cols;
    for (size_t i = 0; i < P * N; i++)
        if (table[i] >= t) return fail(WALLY_EINVAL, "table coefficient %zu is not below t", i);
    uint32_t levels = 0, levels2 = 0;
    while ((1u << levels) < rows) levels++;
    while ((1u << levels2) < rows + cols) levels2++;
    if (levels2 > 12) levels2 = 0;  // the two-dimensional query needs rows + cols <= 4096
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    c->pir_rows = c->pir_cols = c->pir_levels = 0;
    c->pir_db.release();
    DevBuf<u64> raw;
    if (raw.ensure(P * N) != cudaSuccess || c->pir_db.ensure(P * L * N) != cudaSuccess ||
        c->pir_mono.ensure(std::max<size_t>(std::max(levels, levels2), 1) * L * N) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the PIR table (%.2f GB)", P * L * N * 8.0 / 1e9);
    CUDA_TRY(cudaMemcpyAsync(raw.p, table, 8 * P * N, cudaMemcpyHostToDevice, st));
    CUDA_TRY(launch_pir_lift(c->dp, raw.p, (u32)P, c->pir_db.p, st));
    CUDA_TRY(launch_to_ntt(c->dp, nullptr, c->pir_db.p, L * N, c->pir_db.p, L * N, (u32)L, (u32)L, (u32)P, nullptr,
                           true, st));
    // X^(-2^a) = -X^(N - 2^a): its NTT per limb, times 2^64
    const uint32_t lmax = std::max(levels, levels2);
    std::vector<uint64_t> mono(std::max<size_t>(lmax, 1) * L * N, 0);
    for (uint32_t a = 0; a < lmax; a++)
        for (size_t l = 0; l < L; l++) mono[((size_t)a * L + l) * N + (N - (1u << a))] = c->mods[l] - 1;
    if (lmax) {
        CUDA_TRY(cudaMemcpyAsync(c->pir_mono.p, mono.data(), 8 * mono.size(), cudaMemcpyHostToDevice, st));
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, c->pir_mono.p, L * N, c->pir_mono.p, L * N, (u32)L, (u32)L, lmax,
                               nullptr, true, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    raw.release();
    c->pir_rows = rows;
    c->pir_cols = cols;
    c->pir_levels = levels;
    c->pir_levels2 = levels2;
    return WALLY_OK;
}

int wally_pir_answer(wally_ctx *c, uint32_t n, const uint64_t *queries, const uint64_t *keys, uint64_t *out,
                     void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (!c->pir_rows) return fail(WALLY_ESTATE, "no PIR table loaded");
    if (n == 0) return WALLY_OK;
    if (!queries || !out || (c->pir_levels && !keys)) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t lv = c->pir_levels, cols = c->pir_cols, rows = c->pir_rows;
    const size_t L = c->L, ctw = c->ctw(), keyw = c->keysw() / 2;
    const uint32_t chunk = std::min<uint32_t>(n, 64), full = 1u << lv;
    int rc0 = pir_scratch(c, chunk, lv, cols);
    if (rc0) return rc0;
    for (uint32_t q0 = 0; q0 < n; q0 += chunk) {
        const uint32_t nq = std::min(chunk, n - q0);
        // queries and keys to NTT form (keys times 2^64)
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, queries + (size_t)q0 * ctw, ctw, c->pir_E[0].p, ctw, 2 * (u32)L,
                               (u32)L, nq, nullptr, false, st));
        const uint32_t nkeys = lv - pir_key_base(c, lv);
        if (lv)
            CUDA_TRY(launch_to_ntt(c->dp, nullptr, keys + (size_t)q0 * nkeys * keyw, keyw, c->pir_keys.p, keyw,
                                   2 * (u32)(L * (L + 1)), (u32)(L + 1), nq * nkeys, nullptr, true, st));
        int cur = 0;
        int rc = pir_expand(c, nq, lv, cur, st);
        if (rc) return rc;
        CUDA_TRY(launch_pir_dim1(c->dp, c->pir_db.p, rows, cols, c->pir_E[cur].p, full, nq, c->pir_out.p, st));
        CUDA_TRY(launch_from_ntt(c->dp, c->pir_out.p, out + (size_t)q0 * cols * ctw, 2 * (u32)L, (u32)L, nq * cols,
                                 st));
    }
    return WALLY_OK;
}

// ---------------------------------------------------------------- MulPIR's second dimension
namespace {

uint32_t bitlen_big(const std::vector<uint64_t> &a)
{
    for (size_t i = a.size(); i-- > 0;)
        if (a[i]) return (uint32_t)(64 * i + 64 - __builtin_clzll(a[i]));
    return 0;
}

bool to_words(const std::vector<uint64_t> &a, u64 *out)
{
    for (int i = 0; i < XW; i++) out[i] = 0;
    for (size_t i = 0; i < a.size(); i++) {
        if (i >= (size_t)XW) {
            if (a[i]) return false;
            continue;
        }
        out[i] = a[i];
    }
    return true;
}

// The extension basis of the exact tensor: further primes = 1 mod 2N below
// P until their product exceeds 2^(12 + log2 N) Q (twice the largest
// coefficient of a sum of up to 4096 tensors of centred lifts), its own
// context (transform tables) and the CRT constants.
int build_ext(wally_ctx *c)
{
    if (c->ext) return WALLY_OK;
    const uint32_t L = c->L;
    std::vector<uint64_t> Qw{1};
    for (uint32_t i = 0; i < L; i++) Qw = big_mul_small(Qw, c->mods[i]);
    const uint32_t need = bitlen_big(Qw) + c->log_n + 13;
    std::vector<uint64_t> b;
    uint32_t bits = 0;
    uint64_t below = c->mods[L];
    while (bits <= need) {
        below = prime_1mod_below(below, 2 * (uint64_t)c->N);
        if (!below) return fail(WALLY_EINVAL, "no extension primes");
        b.push_back(below);
        bits += 63 - __builtin_clzll(below);
    }
    const uint32_t Lr = L + (uint32_t)b.size();
    if (Lr >= WALLY_MAX_LIMBS)
        return fail(WALLY_EINVAL, "ciphertext products need %u limbs in the extension basis (at most %d)", Lr,
                    WALLY_MAX_LIMBS - 1);
    ExtConst ec;
    memset(&ec, 0, sizeof(ec));
    ec.L = (int)L;
    ec.Lx = (int)b.size();
    ec.Lr = (int)Lr;
    ec.t = c->mods[L + 1];
    std::vector<uint64_t> Rw = Qw;
    for (uint64_t x : b) Rw = big_mul_small(Rw, x);
    bool ok = to_words(Qw, ec.Q) && to_words(Rw, ec.R);
    std::vector<uint64_t> twoQ = big_mul_small(Qw, 2);
    twoQ[0] -= 1;  // 2Q is even and its low word nonzero (Q odd)
    ok = ok && to_words(twoQ, ec.twoQm1);
    for (uint32_t i = 0; i < L; i++) {
        ec.q[i] = c->mods[i];
        ec.theta[i] = c->dp.theta[i];
        uint64_t rem;
        std::vector<uint64_t> qi = big_div_small(Qw, c->mods[i], &rem);
        ok = ok && to_words(qi, ec.qw[i]);
        for (size_t k = 0; k < b.size(); k++) ec.qdiv_b[i][k] = big_mod_small(qi, b[k]);
    }
    for (size_t k = 0; k < b.size(); k++) {
        ec.b[k] = b[k];
        ec.Q_b[k] = big_mod_small(Qw, b[k]);
    }
    for (uint32_t l = 0; l < Lr; l++) {
        const uint64_t r = l < L ? c->mods[l] : b[l - L];
        ec.r[l] = r;
        uint64_t rem;
        std::vector<uint64_t> rl = big_div_small(Rw, r, &rem);
        ok = ok && to_words(rl, ec.rw[l]);
        ec.rinv[l] = invmod_h(big_mod_small(rl, r), r);
    }
    if (!ok) return fail(WALLY_EINVAL, "extension basis wider than %d words", XW);
    std::vector<uint64_t> rq(ec.r, ec.r + Lr);
    wally_params e;
    memset(&e, 0, sizeof(e));
    e.log_n = c->log_n;
    e.num_q = Lr;
    e.q_bits = 61;
    e.t_bits = 30;
    e.dim = c->d;
    e.device = c->device;
    e.q = rq.data();
    e.t = c->mods[L + 1];
    wally_ctx *x = nullptr;
    int rc = wally_setup_params(&e, &x);
    if (rc) return rc;
    if (c->ext_const.ensure(1) != cudaSuccess) {
        wally_destroy(x);
        return fail(WALLY_ENOMEM, "extension constants");
    }
    CUDA_TRY(cudaMemcpy(c->ext_const.p, &ec, sizeof(ec), cudaMemcpyHostToDevice));
    c->ext = x;
    return WALLY_OK;
}

}  // namespace

int wally_keygen_relin(wally_ctx *c, uint32_t n, const int8_t *secret, const uint64_t *key_a, const int8_t *key_e,
                       uint64_t *keys, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !key_a || !key_e || !keys) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_relinkey(c->dp, secret, key_a, key_e, n, keys, (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_pir_answer2(wally_ctx *c, uint32_t n, const uint64_t *queries, const uint64_t *keys,
                      const uint64_t *relin_keys, uint64_t *out, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (!c->pir_rows) return fail(WALLY_ESTATE, "no PIR table loaded");
    if (!c->pir_levels2) return fail(WALLY_EINVAL, "rows + columns must be at most 4096");
    if (n == 0) return WALLY_OK;
    if (!queries || !keys || !relin_keys || !out) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    int rc = build_ext(c);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t lv = c->pir_levels2, cols = c->pir_cols, rows = c->pir_rows;
    const size_t N = c->N, L = c->L, ctw = c->ctw(), keyw = c->keysw() / 2;
    const uint32_t Lr = c->ext->L, full = 1u << lv;
    const uint32_t chunk = std::min<uint32_t>(n, 64);
    rc = pir_scratch(c, chunk, lv, cols);
    if (rc) return rc;
    const size_t ext_ct = (size_t)2 * Lr * N;
    if (c->pd_first.ensure((size_t)chunk * cols * ctw) != cudaSuccess ||
        c->pd_col.ensure((size_t)chunk * cols * ctw) != cudaSuccess ||
        c->pd_A.ensure((size_t)chunk * cols * ext_ct) != cudaSuccess ||
        c->pd_B.ensure((size_t)chunk * cols * ext_ct) != cudaSuccess ||
        c->pd_T.ensure((size_t)chunk * 3 * Lr * N) != cudaSuccess || c->pd_X.ensure((size_t)chunk * ctw) != cudaSuccess ||
        c->pd_add.ensure((size_t)chunk * ctw) != cudaSuccess || c->pd_out.ensure((size_t)chunk * ctw) != cudaSuccess ||
        c->pd_rlk.ensure((size_t)chunk * keyw) != cudaSuccess)
        return fail(WALLY_ENOMEM, "cannot allocate the second-dimension scratch");
    const ExtConst *ec = c->ext_const.p;
    for (uint32_t q0 = 0; q0 < n; q0 += chunk) {
        const uint32_t nq = std::min(chunk, n - q0);
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, queries + (size_t)q0 * ctw, ctw, c->pir_E[0].p, ctw, 2 * (u32)L,
                               (u32)L, nq, nullptr, false, st));
        const uint32_t nkeys = lv - pir_key_base(c, lv);
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, keys + (size_t)q0 * nkeys * keyw, keyw, c->pir_keys.p, keyw,
                               2 * (u32)(L * (L + 1)), (u32)(L + 1), nq * nkeys, nullptr, true, st));
        int cur = 0;
        rc = pir_expand(c, nq, lv, cur, st);
        if (rc) return rc;
        // first dimension over the row indicators, then both operands of the
        // second dimension in coefficient form: the column sums and the
        // column indicators (indicators rows .. rows + cols - 1)
        CUDA_TRY(launch_pir_dim1(c->dp, c->pir_db.p, rows, cols, c->pir_E[cur].p, full, nq, c->pir_out.p, st));
        CUDA_TRY(launch_from_ntt(c->dp, c->pir_out.p, c->pd_first.p, 2 * (u32)L, (u32)L, nq * cols, st));
        for (uint32_t q = 0; q < nq; q++)
            CUDA_TRY(launch_from_ntt(c->dp, c->pir_E[cur].p + ((size_t)q * full + rows) * ctw,
                                     c->pd_col.p + (size_t)q * cols * ctw, 2 * (u32)L, (u32)L, cols, st));
        // exact tensor in the extension basis, summed over the columns
        CUDA_TRY(launch_lift_ext(ec, c->pd_first.p, nq * cols * 2, (u32)N, c->pd_A.p, st));
        CUDA_TRY(launch_lift_ext(ec, c->pd_col.p, nq * cols * 2, (u32)N, c->pd_B.p, st));
        CUDA_TRY(launch_to_ntt(c->ext->dp, nullptr, c->pd_A.p, Lr * N, c->pd_A.p, Lr * N, Lr, Lr, nq * cols * 2,
                               nullptr, false, st));
        CUDA_TRY(launch_to_ntt(c->ext->dp, nullptr, c->pd_B.p, Lr * N, c->pd_B.p, Lr * N, Lr, Lr, nq * cols * 2,
                               nullptr, false, st));
        CUDA_TRY(launch_tensor_acc(ec, c->pd_A.p, c->pd_B.p, nq, cols, (u32)N, c->pd_T.p, st));
        CUDA_TRY(launch_from_ntt(c->ext->dp, c->pd_T.p, c->pd_T.p, 3 * Lr, Lr, nq, st));
        // one rescaling, then one relinearisation: (c0, c2) key-switched from
        // s^2 to s (Rot with the identity automorphism) plus (0, c1)
        CUDA_TRY(launch_scale_ext(ec, c->pd_T.p, nq, (u32)N, c->pd_X.p, c->pd_add.p, st));
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, c->pd_X.p, ctw, c->pd_X.p, ctw, 2 * (u32)L, (u32)L, nq, nullptr, false,
                               st));
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, c->pd_add.p, ctw, c->pd_add.p, ctw, 2 * (u32)L, (u32)L, nq, nullptr,
                               false, st));
        CUDA_TRY(launch_to_ntt(c->dp, nullptr, relin_keys + (size_t)q0 * keyw, keyw, c->pd_rlk.p, keyw,
                               2 * (u32)(L * (L + 1)), (u32)(L + 1), nq, nullptr, true, st));
        RotArgs r;
        memset(&r, 0, sizeof(r));
        r.src = c->pd_X.p;
        r.src_stride = ctw;
        r.dst = c->pd_out.p;
        r.dst_stride = ctw;
        r.add = c->pd_add.p;
        r.add_stride = ctw;
        r.key = c->pd_rlk.p;
        r.key_stride = keyw;
        r.n_max = nq;
        r.galois = 1;
        r.sc = c->pir_sc.p;
        r.dg = c->pir_dg.p;
        r.u = c->pir_u.p;
        r.dd = c->pir_dd.p;
        CUDA_TRY(launch_rotate(c->dp, r, st, c->pr()));
        CUDA_TRY(launch_from_ntt(c->dp, c->pd_out.p, out + (size_t)q0 * ctw, 2 * (u32)L, (u32)L, nq, st));
    }
    return WALLY_OK;
}

int wally_pir_derive_keys(wally_ctx *c, int enable)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    c->pir_derive = enable != 0;
    return WALLY_OK;
}

int wally_pir_key_levels(const wally_ctx *c, int two_dims, uint32_t *first, uint32_t *count)
{
    if (!c || !first || !count) return fail(WALLY_EINVAL, "null argument");
    if (!c->pir_rows) return fail(WALLY_ESTATE, "no PIR table loaded");
    const uint32_t lv = two_dims ? c->pir_levels2 : c->pir_levels;
    if (two_dims && !lv) return fail(WALLY_EINVAL, "rows + columns must be at most 4096");
    *first = pir_key_base(c, lv);
    *count = lv - *first;
    return WALLY_OK;
}

int wally_keygen_galois(wally_ctx *c, uint32_t n, uint32_t nk, const uint64_t *galois, const int8_t *secret,
                        const uint64_t *key_a, const int8_t *key_e, uint64_t *keys, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0 || nk == 0) return WALLY_OK;
    if (nk > 16) return fail(WALLY_EINVAL, "at most 16 keys at a time");
    if (!galois || !secret || !key_a || !key_e || !keys) return fail(WALLY_EINVAL, "null argument");
    KinvList kl;
    memset(&kl, 0, sizeof(kl));
    kl.nk = (int)nk;
    const uint64_t two_n = 2 * (uint64_t)c->N;
    for (uint32_t i = 0; i < nk; i++) {
        if ((galois[i] & 1) == 0 || galois[i] >= two_n) return fail(WALLY_EINVAL, "Galois element %u invalid", i);
        kl.v[i] = inv_mod_2n(galois[i], two_n);
    }
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_keygen_list(c->dp, secret, key_a, key_e, n, kl, keys, (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_encrypt_poly(wally_ctx *c, uint32_t n, const int8_t *secret, const uint64_t *m, const uint64_t *enc_a,
                       const int8_t *enc_e, uint64_t *cts, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !m || !enc_a || !enc_e || !cts) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_encrypt(c->dp, secret, m, enc_a, enc_e, n, cts, (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_decrypt_poly(wally_ctx *c, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                       const uint64_t *cts, int64_t *coeffs, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !cts || !coeffs) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->tmp.ensure((size_t)n * c->L * c->N) != cudaSuccess) return fail(WALLY_ENOMEM, "temporary");
    CUDA_TRY(launch_decrypt_coeffs(c->dp, secret, secret_index, cts, n, c->tmp.p, coeffs, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return WALLY_OK;
}

int wally_sync(wally_ctx *c, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    DeviceGuard guard(c->device);
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t err = 0;
    CUDA_TRY(cudaMemcpy(&err, c->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        CUDA_TRY(cudaMemset(c->d_err, 0, 4));
        return fail(WALLY_EINVAL, "a query named a cluster id out of range");
    }
    return WALLY_OK;
}

int wally_profile_enable(wally_ctx *c, int enable)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    c->prof.reset();
    c->prof.reset_waves();
    c->prof_on = enable != 0;
    return WALLY_OK;
}

int wally_profile_waves(wally_ctx *c, uint32_t cap, uint32_t *call, uint32_t *queries, float *done_ms,
                        uint32_t *count)
{
    if (!c || !count) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(cudaDeviceSynchronize());
    uint32_t n = 0;
    for (const auto &w : c->prof.waves) {
        if (n < cap) {
            float t = 0;
            CUDA_TRY(cudaEventElapsedTime(&t, c->prof.call_start[w.call], w.done));
            if (call) call[n] = w.call;
            if (queries) queries[n] = w.queries;
            if (done_ms) done_ms[n] = t;
        }
        n++;
    }
    c->prof.reset_waves();
    *count = n;
    return WALLY_OK;
}

int wally_profile_read(wally_ctx *c, wally_kernel_time *out, uint32_t cap, uint32_t *count)
{
    static const char *names[KK_COUNT] = {"to_ntt", "ks_a", "ks_b", "ks_c", "mac", "output", "plan", "encode"};
    if (!c || !count) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(cudaDeviceSynchronize());
    double ms[KK_COUNT] = {};
    uint64_t launches[KK_COUNT] = {};
    for (auto &r : c->prof.recs) {
        float t = 0;
        CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.kind] += t;
        launches[r.kind]++;
    }
    c->prof.reset();
    uint32_t n = 0;
    for (int k = 0; k < KK_COUNT; k++) {
        if (!launches[k]) continue;
        if (out && n < cap) {
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, names[k], sizeof(out[n].name) - 1);
            out[n].launches = launches[k];
            out[n].total_ms = ms[k];
        }
        n++;
    }
    *count = n;
    return WALLY_OK;
}

int wally_compress_responses(wally_ctx *c, uint32_t n, const uint64_t *cts, uint8_t *out, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!cts || !out) return fail(WALLY_EINVAL, "null argument");
    if (c->bits0 > 57 || c->bits1 > 57) return fail(WALLY_EINVAL, "response limb too wide to pack");
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_compress(c->dp, cts, n, out, c->drop0, c->drop1, c->bits0, c->bits1, (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_decrypt_compressed(wally_ctx *c, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                             const uint8_t *packed, int64_t *scores, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !packed || !scores) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_decrypt_compressed(c->dp, secret, secret_index, packed, n, c->drop0, c->drop1, c->bits0,
                                       c->bits1, scores, (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_keygen(wally_ctx *c, uint32_t n, const int8_t *secret, const uint64_t *key_a, const int8_t *key_e,
                 uint64_t *keys, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !key_a || !key_e || !keys) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    CUDA_TRY(launch_keygen(c->dp, secret, key_a, key_e, n, c->k1, c->kg, c->k1_inv, c->kg_inv, keys,
                           (cudaStream_t)stream));
    return WALLY_OK;
}

int wally_encrypt_query(wally_ctx *c, uint32_t n, const int8_t *secret, const int8_t *queries, const uint64_t *enc_a,
                        const int8_t *enc_e, uint64_t *cts, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !queries || !enc_a || !enc_e || !cts) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // the temporary is shared by the client calls of this context: order them
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->tmp.ensure((size_t)n * c->N) != cudaSuccess) return fail(WALLY_ENOMEM, "temporary");
    CUDA_TRY(launch_encode_queries(c->dp, queries, n, c->tmp.p, st));
    CUDA_TRY(launch_encrypt(c->dp, secret, c->tmp.p, enc_a, enc_e, n, cts, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return WALLY_OK;
}

int wally_decrypt_scores(wally_ctx *c, uint32_t n, const int8_t *secret, const uint32_t *secret_index,
                         const uint64_t *cts, int64_t *scores, void *stream)
{
    if (!c) return fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!secret || !cts || !scores) return fail(WALLY_EINVAL, "null argument");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(st));
    if (c->tmp.ensure((size_t)n * c->L * c->N) != cudaSuccess) return fail(WALLY_ENOMEM, "temporary");
    CUDA_TRY(launch_decrypt(c->dp, secret, secret_index, cts, n, c->tmp.p, scores, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return WALLY_OK;
}

}  // extern "C"

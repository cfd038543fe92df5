// Device pieces shared by the batched number-count kernels (count.cu: the CUDA-core
// accumulation; count_tc.cu: the tensor-core accumulation): PTX wrappers for mbarriers,
// TMA and tensor memory, the work-item decomposition, the staged copies of one SFT chunk,
// the exact FP64 decision near rounding boundaries and the per-CTA toplist buffers.
#pragma once

#include <cuda.h>

#include "bsh_internal.cuh"
#include "select.cuh"

namespace bsh {
namespace {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait on an mbarrier phase: false after `limit` polls (2^22 by default: seconds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

// Tensor memory (TMEM) holds the per-thread Kahan sums of the weighted counts, which
// leaves shared memory to the staged chunks.  One warp allocates the CTA's columns and
// frees them on every exit path; a warp reaches the 32 TMEM lanes of its quarter
// (warp index mod 4), each thread its own lane, with the 32x32b shape.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// ------------------------------------------------------------ items
struct Item {
    int q, s, fb, bt;
};

// Item order inside a problem: sky points in turn (so a sky patch, a contiguous run of sky
// points, is a contiguous run of items); inside a sky point, binary tiles, then f0 blocks
// (fastest).
__device__ __forceinline__ Item decode_item(const CountArgs& a, long long it) {
    int q = 0;
    while (q + 1 < a.n_probs && it >= a.probs[q + 1].item_begin) ++q;
    const ProbDev& P = a.probs[q];
    const long long loc = it - P.item_begin;
    const long long per_s = (long long)P.n_fb * P.n_bt;
    Item r;
    r.q = q;
    r.s = (int)(loc / per_s);
    const int rem = (int)(loc - (long long)r.s * per_s);
    r.bt = rem / P.n_fb;
    r.fb = rem - r.bt * P.n_fb;
    return r;
}

// Work of the batched kernels.  CTAs c + m * pools (m < pool_size, c < pools) share pool c: a
// contiguous, cost-balanced range [base, base + len) of the item list, walked in a fixed order
// (below), from which its CTAs take one item at a time with an atomic counter.  Of the two CTAs
// resident on an SM, the warp schedulers favour one; with fixed ranges the favoured one
// finishes early and the other runs on alone at a fraction of the SM's issue rate.  A pool
// mixes early CTAs (low block indices) with late ones, and its CTAs end together.
//
// The walk covers the range in sweeps of P items (one sky point's binary tiles and f0
// blocks).  Sweep j covers the items [base + jP, base + (j+1)P), started at offset r (the
// first tile of the next sky point) and wrapped round, so every pool of a problem meets
// binary tile t at about the same time and the tile's orbit rows are read from DRAM about
// once per sweep instead of once per sky point.  A last, partial sweep of m < P items that
// does not reach the next sky point (m <= r) holds tiles [P - r, P - r + m) of one sky point:
// it starts at the tile that is a multiple of m, so that at step x of that sweep every such
// pool is on the tile of residue x mod m (one of two tiles), and the pools whose last sweep
// wraps are on tile x or x + P - m.  r = 0 walks the range in order.
struct Walk {
    long long base, len;
    long long P;
    long long r;
};

// Pool of this CTA and its member index (0 ... pool_size - 1) in the pool.
__device__ __forceinline__ int cta_pool(const CountArgs& a, int* member) {
    const int c = (int)blockIdx.x;
    *member = c / a.pools;
    return c - *member * a.pools;
}

__device__ __forceinline__ Walk pool_walk(const CountArgs& a, int q) {
    Walk w;
    w.base = a.pool_item[q];
    w.len = a.pool_item[q + 1] - w.base;
    w.r = a.pool_sweep[2 * q];
    w.P = a.pool_sweep[2 * q + 1];
    return w;
}

// Item of step k (0 <= k < len) of the walk.
__device__ __forceinline__ long long walk_item(const Walk& w, long long k) {
    if (w.r == 0) return w.base + k;
    const long long j = k / w.P, i = k - j * w.P;
    const long long m = w.len - j * w.P < w.P ? w.len - j * w.P : w.P;   // items in this sweep
    const long long e = m > w.r ? m - w.r : 0;                         // of them at offsets >= r
    if (e == 0 && m < w.P) {                                           // partial, inside one sky point
        const long long rho = (m - (w.P - w.r) % m) % m;
        const long long o = i + rho < m ? i + rho : i + rho - m;
        return w.base + j * w.P + o;
    }
    return w.base + j * w.P + (i < e ? w.r + i : i - e);
}

__host__ __device__ __forceinline__ int align128(int x) { return (x + 127) & ~127; }

constexpr int SCAP = 8;   // deferred near-boundary entries per thread and SFT chunk

// Row stride (32-bit words) of the staged c_q rows: the chunk plus four words, so that
// threads of a warp reading one SFT of up to 8 consecutive orbit rows hit distinct
// shared-memory banks (the TMA box of the table is this wide; a 256-SFT chunk, at the
// box limit, is not padded).
__host__ __device__ __forceinline__ int c_stride(int I) { return I < 256 ? I + 4 : I; }

struct TopSmem {
    unsigned long long tau;
    int count;
    int have_tau;
    float mean, inv_sig;
    int abort;
    // batched kernels: the walk steps this CTA has taken from its pool, a ring indexed by the
    // CTA's item number (written by the one thread issuing a stage, read by all after a barrier)
    long long q_step[4];
    int q_tail;                  // items taken so far
    int q_done;                  // the pool has no items left
};

// Per-item constants shared by every thread.
struct ItemCtx {
    int q, s, fb, bt, j0, jb, c0, pbase, ot0, nrows, F2a, F2r, region, nchunks;
    uint32_t lid_base;
};

__device__ __forceinline__ ItemCtx item_ctx(const CountArgs& a, const Item& it, int THREADS) {
    const ProbDev& P = a.probs[it.q];
    ItemCtx c;
    c.q = it.q;
    c.s = it.s;
    c.fb = it.fb;
    c.bt = it.bt;
    c.j0 = it.fb * P.JB;
    c.jb = imin(P.JB, P.n_f0 - c.j0);
    const int Gj0 = P.G0 + c.j0;
    int lo_bin = Gj0 + P.o_min - 1 - P.k_lo;
    lo_bin = lo_bin < 0 ? 0 : lo_bin;
    c.c0 = (lo_bin >> 5) & ~3;
    c.pbase = Gj0 - P.k_lo - 32 * c.c0;
    const int b0 = it.bt * THREADS;
    const int b1 = imin(b0 + THREADS, P.B) - 1;
    c.ot0 = P.brow[b0];
    c.nrows = P.brow[b1] - c.ot0 + 1;
    c.F2a = (int)llrint(2.0 * P.F0) + 2 * c.j0;
    c.F2r = c.F2a + 2 * ((c.jb - 1) / 2);   // 2 F of the block's middle template (LUT reference)
    const int patch = P.patch_of_s[it.s];
    c.region = P.region_base + patch;
    c.lid_base = (uint32_t)((long long)(it.s - (int)P.patch_start[patch]) * P.B);
    c.nchunks = (P.N + a.chunk - 1) / a.chunk;
    return c;
}

// Sequence number of the stage whose copies are in flight into buffer b, or -1: entries
// 2 and 3 of the `done` words.
template <class StageLayout>
__device__ __forceinline__ int* inflight_slots(unsigned char* smem, const StageLayout& L) {
    return reinterpret_cast<int*>(smem + L.done) + 2;
}

// Issues the TMA / bulk copies of chunk `ch` of item `c` into buffer `buf` of the staging
// layout L (offsets pk, vn, w, c of the two buffers, bar and done); `seq` is the
// stage's sequence number within the CTA.  The stage numbered a.skip_stage (a test hook,
// normally -1) is left unissued: nothing completes its barrier phase, so the wait on it
// expires.
template <class StageLayout>
__device__ __forceinline__ void issue_stage(const CountArgs& a, const TmapSet& maps, const ItemCtx& c, int ch,
                                            unsigned char* smem, const StageLayout& L, int buf, int seq) {
    int* inflight = inflight_slots(smem, L);
    if (seq == a.skip_stage) {
        inflight[buf] = -1;
        return;
    }
    inflight[buf] = seq;
    const ProbDev& P = a.probs[c.q];
    const int I = a.chunk;
    const int i0 = ch * I;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar) + buf;
    // the c_q box holds P.crows rows from the item's first row (rows past the table
    // are zero-filled and still count toward the expected bytes)
    const uint32_t bytes = (uint32_t)(I * a.wseg_max * 4 + I * 4 * 2 + c_stride(I) * P.crows * 4);
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_2d(smem + L.pk[buf], maps.map[c.q], bar, c.c0, i0);
    tma_load_2d(smem + L.c[buf], maps.cmap[c.q], bar, i0, c.ot0);
    bulk_load(smem + L.vn[buf], P.vn_q + (size_t)c.s * P.Np + i0, (uint32_t)(I * 4), bar);
    bulk_load(smem + L.w[buf], P.w32 + (size_t)c.s * P.Np + i0, (uint32_t)(I * 4), bar);
}

// Template-by-template decision of one block at one SFT (rare): the ends are near a
// rounding boundary; FP64 decides the templates within 31 M of it.
__device__ __forceinline__ uint32_t slow_window_exact(const ProbDev& P, int v0, int v1, int pbase, int pos_max,
                                                   const uint32_t* row, int s, int b, int i, int j0,
                                                   unsigned* status) {
    bool have = false;
    double D = 0.0;
    auto exact_o = [&](int j) -> int {
        if (!have) {
            const double* n = P.sky + 3 * (size_t)s;
            const double* v = P.v + 3 * (size_t)i;
            const double vn = __dadd_rn(__dadd_rn(__dmul_rn(v[0], n[0]), __dmul_rn(v[1], n[1])),
                                        __dmul_rn(v[2], n[2]));
            const double c = P.c64[(size_t)P.brow[b] * P.Np + i];
            D = __dsub_rn(vn, __dmul_rn(P.bap[b], c));
            have = true;
        }
        const double F = P.F0 + (double)(j0 + j);
        const double x = __dadd_rn(F, __dmul_rn(F, D));
        const double k = floor(__dadd_rn(x, 0.5));
        return (int)((long long)k - (long long)(P.G0 + j0 + j));
    };
    bool bad = false;
    const uint32_t m = fp_window_exact(v0, v1, pbase, pos_max, P.fp.s_y, P.fp.M, row, exact_o, &bad);
    if (bad) set_status(status, ST_RANGE);
    return m;
}

// ------------------------------------------------------------ toplist pieces
template <int THREADS>
__device__ void topk_reduce(const CountArgs& a, Entry* buf, int keep, TopSmem& ts, SelectSmem& sm) {
    const int n = ts.count;
    __syncthreads();
    if (n <= keep) return;
    auto seg = [&](int, const Entry*& base, int& cnt) {
        base = buf;
        cnt = n;
    };
    const unsigned long long tau = cta_kth_largest<THREADS>(1, seg, keep, sm);
    const int m = cta_compact_ge<THREADS>(buf, n, tau, sm);
    if (threadIdx.x == 0) {
        ts.count = m;
        ts.tau = tau;
        ts.have_tau = 1;
    }
    __syncthreads();
}

template <int THREADS>
__device__ void topk_close_visit(const CountArgs& a, int visit, TopSmem& ts, SelectSmem& sm) {
    if (visit < 0) return;
    Entry* buf = a.visit_buf + (size_t)visit * a.cap;
    topk_reduce<THREADS>(a, buf, a.top_k, ts, sm);
    if (threadIdx.x == 0) {
        a.visit_count[visit] = ts.count;
        ts.count = 0;
        ts.have_tau = 0;
        ts.tau = 0ull;
    }
    __syncthreads();
}

// Walk step of the CTA's item number x (x <= items taken so far): takes the next item of the
// pool when x is one past the last taken.  Returns false once the pool is exhausted.
__device__ __forceinline__ bool pool_take(const CountArgs& a, int q, const Walk& w, TopSmem& ts, int x,
                                          long long* step) {
    if (x >= ts.q_tail) {
        if (ts.q_done) return false;
        const long long s = (long long)atomicAdd(a.pool_next + q, 1ull);
        if (s >= w.len) {
            ts.q_done = 1;
            return false;
        }
        ts.q_step[x & 3] = s;
        ts.q_tail = x + 1;
    }
    *step = ts.q_step[x & 3];
    return true;
}

// Chunk `ch + ahead` of the CTA's item sequence from its item number x, taking items from the
// pool as needed (at most two past x): returns false past the pool's end.
__device__ __forceinline__ bool advance_chunk(const CountArgs& a, int q, const Walk& w, TopSmem& ts, int x, int ch,
                                              int ahead, int threads, ItemCtx* out, int* out_ch) {
    ItemCtx c = item_ctx(a, decode_item(a, walk_item(w, ts.q_step[x & 3])), threads);
    int n = ch + ahead;
    while (n >= c.nchunks) {
        n -= c.nchunks;
        ++x;
        long long st;
        if (!pool_take(a, q, w, ts, x, &st)) return false;
        c = item_ctx(a, decode_item(a, walk_item(w, st)), threads);
    }
    *out = c;
    *out_ch = n;
    return true;
}


}  // namespace
}  // namespace bsh

// Number count (Sec. IV.C, Sec. V.A; track of Eq. (15); significance of
// Eq. (25)) with a fused per-patch toplist.
//
// Work decomposition: an item is (problem q, sky point s, f0 block fb of 32
// templates, binary tile bt of THREADS binary templates).  Each thread owns
// one binary template and the 32 f0 templates of the block: for every SFT the
// track of all 32 f0 templates is one contiguous 32-bit window of the
// peakgram row (consecutive f0 bins, offset constant except at most one
// boundary crossing inside the block), so one shared-memory funnel shift
// yields 32 terms.  Unweighted counts accumulate in bit-sliced carry-save
// counters; weighted counts in FP32 per 64-SFT block, Kahan-compensated across
// blocks in sums held in tensor memory (TMEM).  Persistent CTAs walk a static,
// cost-balanced range of items; the peakgram band and the per-SFT tables of each
// SFT chunk are staged into shared memory by TMA (cp.async.bulk.tensor /
// cp.async.bulk) into two buffers, the next chunk loading while one is counted.
//
// The plain form (BSH_MODE_PLAIN) evaluates the FP64 track for every term,
// sums FP64 weights in FP64, and runs once per sky patch.
#include "count_common.cuh"

namespace bsh {
namespace {

// 2 consecutive columns of this thread's lane at taddr and at taddr + 32 (sum, compensation);
// the wait is in the same statement, so no use of the values can move above it.
__device__ __forceinline__ void tmem_ld2x2(uint32_t taddr, float* a, float* c) {
    uint32_t r[4];
    asm volatile(
        "{\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%4];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%5];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
    a[0] = __uint_as_float(r[0]);
    a[1] = __uint_as_float(r[1]);
    c[0] = __uint_as_float(r[2]);
    c[1] = __uint_as_float(r[3]);
}
__device__ __forceinline__ void tmem_st2x2(uint32_t taddr, const float* a, const float* c) {
    asm volatile(
        "{\n\t"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%4], {%0, %1};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%5], {%2, %3};\n\t"
        "tcgen05.wait::st.sync.aligned;\n\t}"
        ::"r"(__float_as_uint(a[0])), "r"(__float_as_uint(a[1])), "r"(__float_as_uint(c[0])),
          "r"(__float_as_uint(c[1])), "r"(taddr), "r"(taddr + 32u)
        : "memory");
}

// Shared-memory layout of the batched kernel: double-buffered TMA stages
// (peakgram band, vn / weight / c table rows), per-warp track values, the
// TMEM address slot, stage barriers and arrival counters, and the
// toplist bookkeeping.
struct Layout {
    int pk[2], vn[2], w[2], c[2], y, cp, ce, sl, tab, bar, done, tm, sel, misc, total;
};

// direct: the C values are formed per term from the staged c_q rows (no per-warp arrays).
__host__ __device__ inline Layout make_layout(int I, int wseg, int ot_max, int wrows, int threads, int acc,
                                              int direct) {
    Layout L;
    const int nw = threads / 32;
    int o = 0;
    for (int b = 0; b < 2; ++b) { L.pk[b] = o; o = align128(o + I * wseg * 4); }
    for (int b = 0; b < 2; ++b) { L.vn[b] = o; o = align128(o + I * 4); }
    for (int b = 0; b < 2; ++b) { L.w[b] = o; o = align128(o + I * 4); }
    for (int b = 0; b < 2; ++b) { L.c[b] = o; o = align128(o + c_stride(I) * ot_max * 4); }
    L.y = o; o = align128(o + nw * I * 8);
    L.cp = o; o = align128(o + (direct ? 0 : nw * I * wrows * 4));
    L.ce = o; o = align128(o + (direct ? 0 : nw * I * wrows * 8));
    L.sl = o; o = align128(o + SCAP * threads);
    L.tab = o; o = align128(o + (acc ? nw * 256 * 4 : 0));
    L.bar = o; o = align128(o + 16);
    L.done = o; o = align128(o + 16);
    L.tm = o; o = align128(o + 16);
    L.sel = o; o = align128(o + (int)sizeof(SelectSmem));
    L.misc = o; o = align128(o + (int)sizeof(TopSmem));
    L.total = o;
    return L;
}

// 8 x 8 bit-matrix transpose: byte u of x is row u (bit k = column k); on
// return byte k holds column k (bit u = bit k of the input's byte u).
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
    uint64_t t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// Exact FP64 fallback of the look-up-table variant: the modulation at the block's
// reference template jr, near a rounding boundary (rare).
__device__ __noinline__ uint32_t slow_window_lut(const ProbDev& P, int pbase, int pos_max, const uint32_t* row,
                                                 int s, int b, int i, int jr, unsigned* status) {
    const double* n = P.sky + 3 * (size_t)s;
    const double* v = P.v + 3 * (size_t)i;
    const double vn = __dadd_rn(__dadd_rn(__dmul_rn(v[0], n[0]), __dmul_rn(v[1], n[1])), __dmul_rn(v[2], n[2]));
    const double c = P.c64[(size_t)P.brow[b] * P.Np + i];
    const double D = __dsub_rn(vn, __dmul_rn(P.bap[b], c));
    const double F = P.F0 + (double)jr;
    const double x = __dadd_rn(F, __dmul_rn(F, D));
    const int o = (int)((long long)floor(__dadd_rn(x, 0.5)) - (long long)(P.G0 + jr));
    const int pos = pbase + o;
    if (pos < 0 || pos > pos_max) {
        set_status(status, ST_RANGE);
        return 0u;
    }
    return row_window(row, pos);
}

// Scores the 32 templates of this thread and appends the ones above the
// running threshold; returns after the CTA-wide bookkeeping.
template <int THREADS>
__device__ void emit_item(const CountArgs& a, const ProbDev& P, const ItemCtx& c, int b, bool bvalid,
                          const float* nw, const uint32_t* nu, int visit, TopSmem& ts, SelectSmem& sm) {
    const int jb = c.jb;
    if (a.dense) {
        if (bvalid) {
            const size_t base = ((size_t)c.s * P.B + b) * P.n_f0 + c.j0;
            int32_t* du = a.dense_unw[c.q];
            float* dw = a.dense_w[c.q];
#pragma unroll
            for (int j = 0; j < JW; ++j)
                if (j < jb) {
                    du[base + j] = (int32_t)nu[j];
                    dw[base + j] = nw[j];
                }
        }
        return;
    }
    Entry* buf = a.visit_buf + (size_t)visit * a.cap;
    const float mean = ts.mean, isg = ts.inv_sig;
    const unsigned long long tau = ts.tau;
    const bool have = ts.have_tau != 0;
    if (bvalid) {
        const uint32_t lid0 = (c.lid_base + (uint32_t)b) * (uint32_t)P.n_f0 + (uint32_t)c.j0;
#pragma unroll
        for (int j = 0; j < JW; ++j) {
            if (j < jb) {
                const float sc = (nw[j] - mean) * isg;
                const unsigned long long key = make_key(sc, lid0 + (uint32_t)j);
                if (!have || key > tau) {
                    const int pos = atomicAdd(&ts.count, 1);
                    Entry e;
                    e.key = key;
                    e.n_w = nw[j];
                    e.n_unw = (int32_t)nu[j];
                    buf[pos] = e;
                }
            }
        }
    }
    __syncthreads();
    if (ts.count > a.cap - THREADS * JW) topk_reduce<THREADS>(a, buf, a.top_k, ts, sm);
}

// ------------------------------------------------------------ batched kernel
// This warp's TMEM columns: the CTA's base (read back from shared memory, so that no
// register holds it through the hot loop), the lanes of the warp's quarter, 64 columns
// per warp sharing that quarter: [+0, +32) sums, [+32, +64) compensations.
__device__ __forceinline__ uint32_t tmem_cols(const volatile uint32_t* slot, int warp) {
    return *slot + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
}

// Kahan-compensated fold of the 64-SFT block sums into the thread's sums held in TMEM.
__device__ __forceinline__ void kahan_fold(float* part, uint32_t tacc) {
    __syncwarp();   // the tcgen05 accesses below are warp-collective
#pragma unroll
    for (int j0 = 0; j0 < JW; j0 += 2) {
        float a[2], c[2];
        tmem_ld2x2(tacc + (uint32_t)j0, a, c);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float y = part[j0 + k] - c[k];
            const float t = a[k] + y;
            c[k] = (t - a[k]) - y;
            a[k] = t;
            part[j0 + k] = 0.f;
        }
        tmem_st2x2(tacc + (uint32_t)j0, a, c);
    }
}

// ACC selects the weighted accumulation: 0 = one predicated FP32 add per term;
// 1 = per 8 SFTs, a warp-private table of the 256 subset sums of their weights
// and one lookup per f0 template (the 8 window masks are bit-transposed so
// that byte j holds template j's 8 bits).
// LUT = true: the look-up-table approximation of Sec. IV.B -- every template of an f0
// block reads the window at the block's reference template's modulation.
// DIRECT = true: each thread forms C_q from its orbit row's staged c_q entry per term
// instead of reading per-warp converted arrays (for banks where few templates share a
// row and those arrays would not fit in shared memory).
template <int THREADS, int NE, int ACC, bool LUT, bool DIRECT>
__global__ void __launch_bounds__(THREADS, 512 / THREADS)
    count_batched(const CountArgs a, const __grid_constant__ TmapSet maps) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int NW = THREADS / 32;
    const Layout L = make_layout(a.chunk, a.wseg_max, a.ot_max, a.wrows, THREADS, ACC, DIRECT ? 1 : 0);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar);
    unsigned* done = reinterpret_cast<unsigned*>(smem + L.done);
    SelectSmem& sm = *reinterpret_cast<SelectSmem*>(smem + L.sel);
    TopSmem& ts = *reinterpret_cast<TopSmem*>(smem + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int I = a.chunk;
    const int wrows = a.wrows;
    int2* yp = reinterpret_cast<int2*>(smem + L.y) + warp * I;       // Z at the reference, margin
    int* cp = reinterpret_cast<int*>(smem + L.cp) + warp * I * wrows;            // C at the reference
    int2* cpe = reinterpret_cast<int2*>(smem + L.ce) + warp * I * wrows;         // C at j0, j0 + 31
    uint8_t* slist = reinterpret_cast<uint8_t*>(smem + L.sl);                     // [SCAP][THREADS]
    float* tab = reinterpret_cast<float*>(smem + L.tab) + warp * 256;

    int member;
    const int pq = cta_pool(a, &member);
    const Walk wk = pool_walk(a, pq);
    if (tid == 0) {   // the CTA's first item
        ts.q_tail = 0;
        ts.q_done = 0;
        long long s0;
        (void)pool_take(a, pq, wk, ts, 0, &s0);
    }
    __syncthreads();
    if (ts.q_tail == 0) return;   // the other CTA of the pool took every item
    int head = 0;                 // this CTA's item number
    long long step = ts.q_step[0];  // walk step of the current item
    int visit = -1;
    int run = a.pool_run[pq];     // run (one region along the pool's walk) of the current item
    const int run_end = a.pool_run[pq + 1];
    int open_run = -1;

    // TMEM for the Kahan sums: 64 columns per warp quarter-slot (256 threads: warps w and
    // w + 4 share lanes, so 128 columns; 128 threads: 64)
    constexpr uint32_t TCOLS = THREADS > 128 ? 128u : 64u;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tm);
    if (warp == 0) tmem_alloc(tslot, TCOLS);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        done[0] = 0u;
        done[1] = 0u;
        inflight_slots(smem, L)[0] = -1;
        inflight_slots(smem, L)[1] = -1;
        ts.count = 0;
        ts.have_tau = 0;
        ts.tau = 0ull;
        ts.abort = 0;
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();

    ItemCtx cur = item_ctx(a, decode_item(a, walk_item(wk, step)), THREADS);
    if (tid == 0) {
        issue_stage(a, maps, cur, 0, smem, L, 0, 0);
        ItemCtx nx;
        int nch;
        if (advance_chunk(a, pq, wk, ts, 0, 0, 1, THREADS, &nx, &nch)) issue_stage(a, maps, nx, nch, smem, L, 1, 1);
    }
    unsigned g = 0;   // chunk sequence number within this CTA

    while (true) {
        const ProbDev& P = a.probs[cur.q];
        const int b = cur.bt * THREADS + tid;
        const bool bvalid = b < P.B;
        const int b_w0 = cur.bt * THREADS + warp * 32;          // first binary of this warp
        const int otw0 = P.brow[imin(b_w0, P.B - 1)];           // first orbit row of this warp
        const int otw1 = P.brow[imin(b_w0 + 31, P.B - 1)];
        const int nrw = otw1 - otw0 + 1;                        // rows this warp needs (<= wrows)
        const int ot = bvalid ? P.brow[b] - otw0 : 0;
        const int orow0 = otw0 - cur.ot0;                       // their offset in the CTA's staged rows
        const int myrow = bvalid ? P.brow[b] - cur.ot0 : 0;      // this thread's staged row (DIRECT)
        const int apq = bvalid ? P.bapq[b] : 0;
        const int s_y = P.fp.s_y, M = P.fp.M;
        const int wseg = a.wseg_max;
        const int pos_max = 32 * wseg - 33;
        const int pbase = cur.pbase;

        // new run of the pool's walk -> new visit buffer (the run's buffer of this member)
        if (!a.dense) {
            while (run + 1 < run_end && step >= a.run_step[run + 1]) ++run;
            if (run != open_run) {
                if (open_run >= 0) topk_close_visit<THREADS>(a, visit, ts, sm);
                visit = a.pool_size * run + member;
                open_run = run;
            }
        }
        if (tid == 0) {
            const double sw = P.sum_w[cur.s], sw2 = P.sum_w2[cur.s];
            const double var = P.p_th * (1.0 - P.p_th) * sw2;
            ts.mean = (float)(P.p_th * sw);
            ts.inv_sig = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.f;
        }

        float part[JW];
#pragma unroll
        for (int j = 0; j < JW; ++j) part[j] = 0.f;
        {
            const float z[2] = {0.f, 0.f};
            const uint32_t tacc = tmem_cols(tslot, warp);
            __syncwarp();
#pragma unroll
            for (int j0 = 0; j0 < JW; j0 += 2) tmem_st2x2(tacc + (uint32_t)j0, z, z);
        }
        uint32_t ones = 0, twos = 0, fours = 0;
        uint32_t e8[NE];   // bit-sliced count of the 'eights' (N < 8 * 2^NE)
#pragma unroll
        for (int k = 0; k < NE; ++k) e8[k] = 0;

        // track values at the reference template (the block's j0 + 15; the LUT's middle template)
        const int F2a = cur.F2a, F2b = cur.F2a + 62, F2ref = LUT ? cur.F2r : cur.F2a + 30;
        const FixedPoint fpl = P.fp;
        bool aborted = false;
        for (int ch = 0; ch < cur.nchunks; ++ch, ++g) {
            const int buf = g & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[buf], (g >> 1) & 1, a.wait_polls))) {   // warp-uniform exit
                if (lane == 0) {
                    set_status(a.status, ST_TIMEOUT);
                    ts.abort = 1;
                }
                aborted = true;
                break;
            }
            // this warp's track values for the chunk: Z at the reference template with the SFT's
            // margin (the slope bound; M alone for the LUT), C_q at the reference template and at
            // the block's ends (Z at the ends is formed from the staged vn_q by the rare deferred
            // entries that need it)
            const int32_t* vnr = reinterpret_cast<const int32_t*>(smem + L.vn[buf]);
            const int32_t* cr = reinterpret_cast<const int32_t*>(smem + L.c[buf]);
            for (int e = lane; e < I; e += 32) {
                const int vq = vnr[e];
                yp[e] = make_int2(make_Z(F2ref, vq, fpl), LUT ? fpl.M : fp_margin(vq, fpl));
            }
            if (!DIRECT) {
                for (int e = lane; e < I * nrw; e += 32) {
                    const int r = e / I, il = e - r * I;
                    const int cq = cr[(orow0 + r) * c_stride(I) + il];
                    cp[il * wrows + r] = make_C(F2ref, cq, fpl);
                    if (!LUT) cpe[il * wrows + r] = make_int2(make_C(F2a, cq, fpl), make_C(F2b, cq, fpl));
                }
            }
            const int32_t* myc = cr + myrow * c_stride(I);
            __syncwarp();
            const uint32_t* pk = reinterpret_cast<const uint32_t*>(smem + L.pk[buf]);
            const float* wt = reinterpret_cast<const float*>(smem + L.w[buf]);
            const int i0 = ch * I;
            int scnt = 0;                 // deferred entries of this thread in this chunk
            for (int g8 = 0; g8 < I; g8 += 8) {
                uint32_t mk[8];
                unsigned slow = 0u;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int il = g8 + u;
                    const int2 z = yp[il];
                    const int cc = DIRECT ? make_C(F2ref, myc[il], fpl) : cp[il * wrows + ot];
                    const int v = z.x - __mulhi(apq, cc);
                    // in the staged segment by construction (host band check, device velocity
                    // check); the clamp only keeps the read in bounds
                    const unsigned pos = min((unsigned)(pbase + (v >> s_y)), (unsigned)pos_max);
                    mk[u] = row_window(pk + il * wseg, (int)pos);
                    slow |= (fp_fast_ref(v, z.y, s_y) ? 0u : 1u) << u;
                }
                if (slow) {       // rare: near a rounding boundary
                    unsigned now = 0u;
                    if (!LUT) {
                        // defer to the chunk's end, where the lanes resolve them together
                        unsigned sl = slow;
                        while (sl) {
                            const int u = __ffs(sl) - 1;
                            sl &= sl - 1u;
                            if (scnt < SCAP) slist[scnt++ * THREADS + tid] = (uint8_t)(g8 + u);
                            else now |= 1u << u;
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            if ((slow >> k) & 1u) mk[k] = 0u;
                    } else {
                        now = slow;
                    }
                    while (now) {
                        const int u = __ffs(now) - 1;
                        now &= now - 1u;
                        const int il = g8 + u;
                        uint32_t wv = 0u;
                        if (bvalid && i0 + il < P.N) {
                            if (LUT) {
                                wv = slow_window_lut(P, pbase, pos_max, pk + il * wseg, cur.s, b, i0 + il,
                                                     cur.j0 + (cur.jb - 1) / 2, a.status);
                            } else {
                                const int2 ze = make_int2(make_Z(F2a, vnr[il], fpl), make_Z(F2b, vnr[il], fpl));
                                const int2 ce = DIRECT ? make_int2(make_C(F2a, myc[il], fpl), make_C(F2b, myc[il], fpl))
                                                       : cpe[il * wrows + ot];
                                const int v0 = ze.x - __mulhi(apq, ce.x);
                                const int v1 = ze.y - __mulhi(apq, ce.y);
                                int path;
                                if (!fp_window_ends(v0, v1, pbase, pos_max, s_y, M, pk + il * wseg, &wv, &path))
                                    wv = slow_window_exact(P, v0, v1, pbase, pos_max, pk + il * wseg, cur.s, b,
                                                           i0 + il, cur.j0, a.status);
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) mk[k] = (k == u) ? wv : mk[k];
                    }
                }
                if (ACC == 0) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const uint32_t m = mk[u];
                        const float wv = wt[g8 + u];
#pragma unroll
                        for (int j = 0; j < JW; ++j)
                            if (m & (1u << j)) part[j] += wv;
                    }
                } else {
                    // subset sums of the 8 weights: entry 32 m + l = low(l) + high(m)
                    const float* wg = wt + g8;
                    float lo = 0.f;
#pragma unroll
                    for (int u = 0; u < 5; ++u)
                        if ((lane >> u) & 1) lo += wg[u];
                    const float w5 = wg[5], w6 = wg[6], w7 = wg[7];
                    const float h3 = w5 + w6;
                    __syncwarp();                 // the previous group's lookups are done
                    tab[lane] = lo;
                    tab[32 + lane] = lo + w5;
                    tab[64 + lane] = lo + w6;
                    tab[96 + lane] = lo + h3;
                    tab[128 + lane] = lo + w7;
                    tab[160 + lane] = lo + (w5 + w7);
                    tab[192 + lane] = lo + (w6 + w7);
                    tab[224 + lane] = lo + (h3 + w7);
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const unsigned sel = (unsigned)q | ((unsigned)(q + 4) << 4);
                        const uint32_t a01 = __byte_perm(mk[0], mk[1], sel);
                        const uint32_t a23 = __byte_perm(mk[2], mk[3], sel);
                        const uint32_t a45 = __byte_perm(mk[4], mk[5], sel);
                        const uint32_t a67 = __byte_perm(mk[6], mk[7], sel);
                        const uint64_t x = transpose8x8(((uint64_t)__byte_perm(a45, a67, 0x5410) << 32) |
                                                        (uint64_t)__byte_perm(a01, a23, 0x5410));
#pragma unroll
                        for (int k = 0; k < 8; ++k) part[8 * q + k] += tab[(unsigned)(x >> (8 * k)) & 0xffu];
                    }
                }
                // (bits of templates past the block or of an invalid binary index are
                // accumulated but never emitted)
                uint32_t tA, tB, fA, fB, eights;
                csa(tA, ones, ones, mk[0], mk[1]);
                csa(tB, ones, ones, mk[2], mk[3]);
                csa(fA, twos, twos, tA, tB);
                csa(tA, ones, ones, mk[4], mk[5]);
                csa(tB, ones, ones, mk[6], mk[7]);
                csa(fB, twos, twos, tA, tB);
                csa(eights, fours, fours, fA, fB);
#pragma unroll
                for (int k = 0; k < NE; ++k) {
                    const uint32_t t = e8[k] & eights;
                    e8[k] ^= eights;
                    eights = t;
                }
                if ((g8 & 63) == 56) kahan_fold(part, tmem_cols(tslot, warp));   // every 64 SFTs
            }
            if (!LUT) {
                // the chunk's deferred entries: each lane its own, all lanes at once
                const int npass = __reduce_max_sync(0xffffffffu, scnt);
                for (int k = 0; k < npass; ++k) {
                    if (k >= scnt) continue;
                    const int il = slist[k * THREADS + tid];
                    uint32_t m = 0u;
                    if (bvalid && i0 + il < P.N) {
                        const int2 ze = make_int2(make_Z(F2a, vnr[il], fpl), make_Z(F2b, vnr[il], fpl));
                        const int2 ce = DIRECT ? make_int2(make_C(F2a, myc[il], fpl), make_C(F2b, myc[il], fpl))
                                               : cpe[il * wrows + ot];
                        const int v0 = ze.x - __mulhi(apq, ce.x);
                        const int v1 = ze.y - __mulhi(apq, ce.y);
                        int path;
                        if (!fp_window_ends(v0, v1, pbase, pos_max, s_y, M, pk + il * wseg, &m, &path))
                            m = slow_window_exact(P, v0, v1, pbase, pos_max, pk + il * wseg, cur.s, b, i0 + il,
                                                  cur.j0, a.status);
                    }
                    const float wv = wt[il];
#pragma unroll
                    for (int j = 0; j < JW; ++j)
                        if (m & (1u << j)) part[j] += wv;
                    // one more mask into the bit-sliced counters
                    uint32_t c = m, t;
                    t = ones & c; ones ^= c; c = t;
                    t = twos & c; twos ^= c; c = t;
                    t = fours & c; fours ^= c; c = t;
#pragma unroll
                    for (int q = 0; q < NE; ++q) {
                        t = e8[q] & c;
                        e8[q] ^= c;
                        c = t;
                    }
                }
            }
            // done with this buffer: the last warp to finish refills it two chunks ahead
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();   // this warp's reads of the buffer precede its arrival
                const unsigned prev = atomicAdd(&done[buf], 1u);
                if (prev == NW * ((g >> 1) + 1) - 1) {
                    __threadfence_block();   // the previous issuer's writes of the item ring
                    ItemCtx nx;
                    int nch;
                    if (advance_chunk(a, pq, wk, ts, head, ch, 2, THREADS, &nx, &nch))
                        issue_stage(a, maps, nx, nch, smem, L, buf, (int)g + 2);
                }
            }
        }
        // fold the last partial block and read out the counts
        const uint32_t tacc = tmem_cols(tslot, warp);
        kahan_fold(part, tacc);
        float nw[JW];
        uint32_t nu[JW];
#pragma unroll
        for (int j0 = 0; j0 < JW; j0 += 2) {
            float sa[2], sc[2];
            tmem_ld2x2(tacc + (uint32_t)j0, sa, sc);
#pragma unroll
            for (int k = 0; k < 2; ++k) nw[j0 + k] = sa[k] - sc[k];
        }
#pragma unroll
        for (int j = 0; j < JW; ++j) {
            uint32_t cnt = ((ones >> j) & 1u) + 2u * ((twos >> j) & 1u) + 4u * ((fours >> j) & 1u);
#pragma unroll
            for (int k = 0; k < NE; ++k) cnt += ((e8[k] >> j) & 1u) << (3 + k);
            nu[j] = cnt;
        }
        (void)aborted;
        if (__syncthreads_or(ts.abort)) break;   // a wait expired somewhere: leave together
        emit_item<THREADS>(a, P, cur, b, bvalid, nw, nu, visit, ts, sm);

        // the last chunk's issuer has taken the next item or found the pool exhausted
        ++head;
        if (head >= ts.q_tail) break;
        step = ts.q_step[head & 3];
        cur = item_ctx(a, decode_item(a, walk_item(wk, step)), THREADS);
        __syncthreads();
    }
    if (!ts.abort && !a.dense && open_run >= 0) topk_close_visit<THREADS>(a, visit, ts, sm);
    // after an expired wait, copies issued into the other buffer may still be landing in this
    // CTA's shared memory: wait (bounded) for every stage still marked in flight before the
    // CTA exits (every warp is past its last issue: they all met at the exit barrier)
    if (ts.abort && tid == 0) {
        const int* inflight = inflight_slots(smem, L);
        for (int bb = 0; bb < 2; ++bb)
            if (inflight[bb] >= 0) (void)mbar_wait(&bars[bb], ((unsigned)inflight[bb] >> 1) & 1u, a.wait_polls);
    }
    // every warp is done with its TMEM columns before the allocating warp frees them
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_free(*tslot, TCOLS);
}

// ------------------------------------------------------------ plain kernel
// FP64 track for every term and FP64 weighted sums; one launch per patch.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) count_plain(const CountArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    SelectSmem& sm = *reinterpret_cast<SelectSmem*>(smem);
    TopSmem& ts = *reinterpret_cast<TopSmem*>(smem + align128((int)sizeof(SelectSmem)));
    const int tid = threadIdx.x;
    long long it = a.cta_item[blockIdx.x];
    const long long it_end = a.cta_item[blockIdx.x + 1];
    if (it >= it_end) return;
    int visit = a.cta_visit[blockIdx.x] - 1;
    int region = -1;
    if (tid == 0) {
        ts.count = 0;
        ts.have_tau = 0;
        ts.tau = 0ull;
    }
    __syncthreads();
    for (; it < it_end; ++it) {
        const ItemCtx cur = item_ctx(a, decode_item(a, it), THREADS);
        const ProbDev& P = a.probs[cur.q];
        const int b = cur.bt * THREADS + tid;
        const bool bvalid = b < P.B;
        if (!a.dense && cur.region != region) {
            if (region >= 0) topk_close_visit<THREADS>(a, visit, ts, sm);
            ++visit;
            region = cur.region;
        }
        if (tid == 0) {
            const double sw = P.sum_w[cur.s], sw2 = P.sum_w2[cur.s];
            const double var = P.p_th * (1.0 - P.p_th) * sw2;
            ts.mean = (float)(P.p_th * sw);
            ts.inv_sig = var > 0.0 ? (float)(1.0 / sqrt(var)) : 0.f;
        }
        double accw[JW];
        uint32_t cnt[JW];
#pragma unroll
        for (int j = 0; j < JW; ++j) { accw[j] = 0.0; cnt[j] = 0u; }
        if (bvalid) {
            const int otg = P.brow[b];
            const double ap = P.bap[b];
            const double* n = P.sky + 3 * (size_t)cur.s;
            for (int i = 0; i < P.N; ++i) {
                const double* v = P.v + 3 * (size_t)i;
                const double vn = __dadd_rn(__dadd_rn(__dmul_rn(v[0], n[0]), __dmul_rn(v[1], n[1])),
                                            __dmul_rn(v[2], n[2]));
                const double D = __dsub_rn(vn, __dmul_rn(ap, P.c64[(size_t)otg * P.Np + i]));
                const double wv = P.w64[(size_t)cur.s * P.Np + i];
                const uint32_t* row = P.bits + (size_t)i * P.W;
#pragma unroll
                for (int j = 0; j < JW; ++j) {
                    if (j < cur.jb) {
                        const double F = P.F0 + (double)(cur.j0 + j);
                        const double x = __dadd_rn(F, __dmul_rn(F, D));
                        const long long k = (long long)floor(__dadd_rn(x, 0.5));
                        const long long col = k - P.k_lo;
                        uint32_t bit = 0u;
                        if (col >= 0 && col < P.K) bit = (__ldg(row + (col >> 5)) >> (col & 31)) & 1u;
                        else set_status(a.status, ST_RANGE);
                        cnt[j] += bit;
                        if (bit) accw[j] = __dadd_rn(accw[j], wv);
                    }
                }
            }
        }
        float nw[JW];
        uint32_t nu[JW];
#pragma unroll
        for (int j = 0; j < JW; ++j) { nw[j] = (float)accw[j]; nu[j] = cnt[j]; }
        __syncthreads();
        emit_item<THREADS>(a, P, cur, b, bvalid, nw, nu, visit, ts, sm);
        __syncthreads();
    }
    if (!a.dense) topk_close_visit<THREADS>(a, visit, ts, sm);
}

}  // namespace

int count_c_stride(int I) { return c_stride(I); }

int count_smem_bytes(int mode, int I, int wseg, int ot_max, int wrows, int threads, int acc, int direct) {
    if (mode == BSH_MODE_PLAIN) return align128((int)sizeof(SelectSmem)) + align128((int)sizeof(TopSmem));
    return make_layout(I, wseg, ot_max, wrows, threads, acc, direct).total;
}

void launch_count(const CountArgs& a, const TmapSet& maps, int grid, int threads, cudaStream_t st) {
    if (grid <= 0) return;
    if (a.mode == BSH_MODE_PLAIN) {
        if (threads == 128) {
            static int s_count_plain128 = 0;
            ensure_smem(count_plain<128>, a.smem_bytes, &s_count_plain128);
            count_plain<128><<<grid, 128, a.smem_bytes, st>>>(a);
        } else {
            static int s_count_plain256 = 0;
            ensure_smem(count_plain<256>, a.smem_bytes, &s_count_plain256);
            count_plain<256><<<grid, 256, a.smem_bytes, st>>>(a);
        }
        return;
    }
    const bool small_n = a.max_n < 8 * 1024;
#define BSH_LAUNCH_BATCHED(T, NE, ACC, LUT, DIR)                                        \
    do {                                                                                \
        static int s_done = 0;                                                          \
        ensure_smem(count_batched<T, NE, ACC, LUT, DIR>, a.smem_bytes, &s_done);        \
        count_batched<T, NE, ACC, LUT, DIR><<<grid, T, a.smem_bytes, st>>>(a, maps);    \
    } while (0)
#define BSH_LAUNCH_ACC(T, NE, LUT)                                                \
    do {                                                                          \
        if (a.direct) BSH_LAUNCH_BATCHED(T, NE, 0, LUT, true);                    \
        else if (a.acc_mode) BSH_LAUNCH_BATCHED(T, NE, 1, LUT, false);            \
        else BSH_LAUNCH_BATCHED(T, NE, 0, LUT, false);                            \
    } while (0)
#define BSH_LAUNCH_NE(T, LUT)                                                     \
    do {                                                                          \
        if (small_n) BSH_LAUNCH_ACC(T, 10, LUT);                                  \
        else BSH_LAUNCH_ACC(T, 13, LUT);                                          \
    } while (0)
    if (threads == 128) {
        if (a.lut) BSH_LAUNCH_NE(128, true); else BSH_LAUNCH_NE(128, false);
    } else {
        if (a.lut) BSH_LAUNCH_NE(256, true); else BSH_LAUNCH_NE(256, false);
    }
#undef BSH_LAUNCH_NE
#undef BSH_LAUNCH_ACC
#undef BSH_LAUNCH_BATCHED
}

}  // namespace bsh

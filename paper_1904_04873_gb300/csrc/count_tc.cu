// Number count (Sec. IV.C; track of Eq. (15); significance of Eq. (25)) with the
// weighted and the unweighted sums formed on the tensor cores (tcgen05.mma).
//
// The count of a block of templates over a block of SFTs is a matrix product:
//   D[t][n] = sum_k A[t][k] B[k][n],
// with A[t][k] = 1 when template t's track hits a peak in SFT k (0 otherwise) and
// B[k][n] the n-th base-16 digit of SFT k's weight in fixed point (w round(2^24 w)),
// n = 0..7, plus a column of ones (n = 8).  Column 8 of D is the unweighted count,
// and sum_n 16^n D[t][n] 2^-24 the weighted count, both exact: every product and
// partial sum is an integer multiple of the smallest A value, far inside FP32's
// exact-integer range, so the accumulation has no rounding at all (fp16 weights are
// integers times 2^-24, so their fixed-point form is exact too).
//
// Work decomposition: an item is (problem, sky point, f0 block of 32 templates, tile
// of 64 binary templates) = 2048 templates = 16 MMA tiles of 128 rows.  One CTA per SM,
// sixteen warps: warp w handles binary templates 32 (w & 1) + lane of the tile and, in
// every K-block of 32 SFTs, the 4 SFTs 4 (w >> 1) .. 4 (w >> 1) + 3.  Per SFT each thread
// forms the 32-bit peak window of its binary template's 32 f0 templates exactly as the
// CUDA-core kernel does (fixed-point track, exact FP64 decision near rounding
// boundaries), and spreads it into 32 bytes of A (e4m3: 0x01 = 2^-9 or 0), stored
// M-major.  A and B are double-buffered: the last warp to store a K-block issues its 16
// MMAs (M = 128, N = 16, K = 32, kind::f8f6f4, D in tensor memory) and commits them to
// the buffer's barrier, and a buffer is stored again once the MMAs of the K-block two
// back have completed, so the windows of one K-block are formed while the tensor cores
// read the previous one.  At the end of an item every thread reads 4 templates' sums
// from tensor memory, forms the counts and the significance and feeds the CTA's toplist
// as the CUDA-core kernel does.
#include "count_common.cuh"

namespace bsh {
namespace {

constexpr int TC_PRODUCERS = 16;                 // warps forming peak windows
constexpr int TC_THREADS = 32 * TC_PRODUCERS;
constexpr int TC_TB = 64;                        // binary templates per item
constexpr int TC_KB = 32;                        // SFTs per K-block (K of one MMA)
constexpr int TC_SLOT = TC_KB / (TC_PRODUCERS / 2);   // SFTs of a K-block per producer warp (4)
constexpr int TC_ROWS = TC_TB * JW;              // 2048 templates per item
constexpr int TC_TILES = TC_ROWS / 128;          // 16 MMA tiles of 128 rows
// A (templates x SFTs of one K-block, one byte each) in the no-swizzle M-major layout:
// 16-row chunks 144 bytes apart (9 x 16 bytes, so that the 16-byte stores of the lanes of
// a quarter-warp land in distinct bank groups), groups of 8 K columns A_LBO bytes apart.
constexpr int A_SBO = 144;
constexpr int A_LBO = (TC_ROWS / 16) * A_SBO;
constexpr int A_BYTES = 4 * A_LBO;               // 72 KB per buffer, two buffers
// B (SFTs x 16 digit columns), N-major: 8-K groups of 8 x 16 bytes, 128 bytes apart
constexpr int B_LBO = 128;
constexpr int B_BYTES = 512;
constexpr uint32_t TC_TCOLS = 16u * TC_TILES;    // 256 tensor-memory columns

struct TcLayout {
    int a[2], b[2], pk[2], vn[2], w[2], c[2], y, cp, ce, bar, mma, done, tm, sel, misc, total;
};

__host__ __device__ inline TcLayout make_tc_layout(int I, int wseg, int ot_max, int wrows, int direct) {
    TcLayout L;
    const int per_warp = I / (TC_KB / TC_SLOT);  // SFTs of one chunk a producer warp forms windows for
    int o = 0;
    for (int b = 0; b < 2; ++b) { L.a[b] = o; o = align128(o + A_BYTES); }
    for (int b = 0; b < 2; ++b) { L.b[b] = o; o = align128(o + B_BYTES); }
    for (int b = 0; b < 2; ++b) { L.pk[b] = o; o = align128(o + I * wseg * 4); }
    for (int b = 0; b < 2; ++b) { L.vn[b] = o; o = align128(o + I * 4); }
    for (int b = 0; b < 2; ++b) { L.w[b] = o; o = align128(o + I * 4); }
    for (int b = 0; b < 2; ++b) { L.c[b] = o; o = align128(o + c_stride(I) * ot_max * 4); }
    L.y = o; o = align128(o + TC_PRODUCERS * per_warp * 8);
    L.cp = o; o = align128(o + (direct ? 0 : TC_PRODUCERS * per_warp * wrows * 4));
    L.ce = o; o = align128(o + (direct ? 0 : TC_PRODUCERS * per_warp * wrows * 8));
    L.bar = o; o = align128(o + 16);
    L.mma = o; o = align128(o + 32);
    L.done = o; o = align128(o + 16);
    L.tm = o; o = align128(o + 16);
    L.sel = o; o = align128(o + (int)sizeof(SelectSmem));
    L.misc = o; o = align128(o + (int)sizeof(TopSmem));
    L.total = o;
    return L;
}

// Shared-memory matrix descriptor, no swizzle: start address, byte offset between core
// matrices along K (leading) and along M / N (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: D in FP32, A and B e4m3, both M/N-major,
// N = 16, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 15) | (1u << 16) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "{\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// e4m3 code of an integer 0..15 (exact).
__device__ __forceinline__ uint32_t e4m3_digit(uint32_t d) {
    if (d == 0u) return 0u;
    const int ex = 31 - __clz((int)d);
    return (uint32_t)(((ex + 7) << 3) | (((d << 3) >> ex) & 7u));
}

// The CTA's weighted and unweighted counts of one item: Eq. (25) scores into the toplist.
// Producer warp w reads tiles t = 4 (w >> 2) + t', t' < 4, at lanes 32 (w & 3) + x; lane x
// of tile t holds byte position p = 16 (t >> 3) + (x & 15) of binary template
// 8 (t & 7) + 2 (w & 3) + (x >> 4) of the item's tile, i.e. its f0 template
// j = (p >> 2) + 8 (p & 3).
__device__ void tc_emit(const CountArgs& a, const ProbDev& P, const ItemCtx& c, uint32_t tbase, int visit,
                        TopSmem& ts, SelectSmem& sm) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const int Q = warp & 3;
        const float mean = ts.mean, isg = ts.inv_sig;
        const unsigned long long tau = ts.tau;
        const bool have = ts.have_tau != 0;
        Entry* buf = a.visit_buf + (size_t)visit * a.cap;
#pragma unroll 1
        for (int tp = 0; tp < 4; ++tp) {
            const int t = 4 * (warp >> 2) + tp;
            float v[16];
            tmem_ld16(tbase + ((uint32_t)(32 * Q) << 16) + (uint32_t)(16 * t), v);
            const int p = 16 * (t >> 3) + (lane & 15);
            const int j = (p >> 2) + 8 * (p & 3);
            const int b = c.bt * TC_TB + 8 * (t & 7) + 2 * Q + (lane >> 4);
            if (b >= P.B || j >= c.jb) continue;
            unsigned long long W = 0ull;
#pragma unroll
            for (int n = 7; n >= 0; --n) W = (W << 4) + (unsigned long long)__float2uint_rn(v[n] * 512.0f);
            const float nw = __ull2float_rn(W) * 5.9604644775390625e-8f;   // x 2^-24
            const uint32_t nu = __float2uint_rn(v[8] * 512.0f);
            if (a.dense) {
                const size_t idx = ((size_t)c.s * P.B + b) * P.n_f0 + c.j0 + j;
                a.dense_unw[c.q][idx] = (int32_t)nu;
                a.dense_w[c.q][idx] = nw;
                continue;
            }
            const float sc = (nw - mean) * isg;
            const uint32_t lid = (c.lid_base + (uint32_t)b) * (uint32_t)P.n_f0 + (uint32_t)(c.j0 + j);
            const unsigned long long key = make_key(sc, lid);
            if (!have || key > tau) {
                const int pos = atomicAdd(&ts.count, 1);
                Entry e;
                e.key = key;
                e.n_w = nw;
                e.n_unw = (int32_t)nu;
                buf[pos] = e;
            }
        }
    }
    __syncthreads();
    if (!a.dense && ts.count > a.cap - TC_ROWS)
        topk_reduce<TC_THREADS>(a, a.visit_buf + (size_t)visit * a.cap, a.top_k, ts, sm);
}

// Expired wait: record it and make the CTA leave at the item's end.
__device__ __forceinline__ void tc_timeout(const CountArgs& a, TopSmem& ts, int lane, bool* abort) {
    if (lane == 0) {
        set_status(a.status, ST_TIMEOUT);
        ts.abort = 1;
    }
    *abort = true;
}

template <bool DIRECT>
__global__ void __launch_bounds__(TC_THREADS, 1) count_tc(const CountArgs a, const __grid_constant__ TmapSet maps) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcLayout L = make_tc_layout(a.chunk, a.wseg_max, a.ot_max, a.wrows, DIRECT ? 1 : 0);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint64_t* a_empty = reinterpret_cast<uint64_t*>(smem + L.mma);   // [2]: a buffer's MMAs are done
    unsigned* a_cnt = reinterpret_cast<unsigned*>(a_empty + 2);        // [2]: warps that stored a buffer
    unsigned* done = reinterpret_cast<unsigned*>(smem + L.done);
    SelectSmem& sm = *reinterpret_cast<SelectSmem*>(smem + L.sel);
    TopSmem& ts = *reinterpret_cast<TopSmem*>(smem + L.misc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = warp & 1;                      // binary group: templates 32 g + lane of the tile
    const int r = warp >> 1;                     // SFT slot: columns 4 r .. 4 r + 3 of each K-block
    const int I = a.chunk;
    const int per_warp = I / (TC_KB / TC_SLOT);
    const int wrows = a.wrows;
    int2* yp = reinterpret_cast<int2*>(smem + L.y) + warp * per_warp;
    int* cp = reinterpret_cast<int*>(smem + L.cp) + warp * per_warp * wrows;
    int2* cpe = reinterpret_cast<int2*>(smem + L.ce) + warp * per_warp * wrows;
    // this thread's two 16-row chunks of A: binary template 32 g + lane, byte positions 0-15 and 16-31;
    // K column 4 r + u lies in group r / 2 of 8 columns, at row 4 (r & 1) + u of it
    const uint32_t a_off0 = (uint32_t)((32 * g + lane) * A_SBO + (r >> 1) * A_LBO + (4 * (r & 1)) * 16);
    const uint32_t a_off1 = a_off0 + (uint32_t)(64 * A_SBO);

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

    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tm);
    if (warp == 0) tmem_alloc(tslot, TC_TCOLS);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&a_empty[0], 1);
        mbar_init(&a_empty[1], 1);
        a_cnt[0] = 0u;
        a_cnt[1] = 0u;
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
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(tslot);

    ItemCtx cur = item_ctx(a, decode_item(a, walk_item(wk, step)), TC_TB);
    if (tid == 0) {
        issue_stage(a, maps, cur, 0, smem, L, 0, 0);
        ItemCtx nx;
        int nch;
        if (advance_chunk(a, pq, wk, ts, 0, 0, 1, TC_TB, &nx, &nch)) issue_stage(a, maps, nx, nch, smem, L, 1, 1);
    }
    unsigned gch = 0;       // chunk sequence number within this CTA
    unsigned kbs = 0;       // K-block sequence number within this CTA
    bool abort = false;

    while (true) {
        const ProbDev& P = a.probs[cur.q];
        if (!a.dense) {   // new run of the pool's walk -> new visit buffer (this member's)
            while (run + 1 < run_end && step >= a.run_step[run + 1]) ++run;
            if (run != open_run) {
                if (open_run >= 0) topk_close_visit<TC_THREADS>(a, visit, ts, sm);
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
        const int b = cur.bt * TC_TB + 32 * g + lane;
        const bool bvalid = b < P.B;
        const int b_w0 = cur.bt * TC_TB + 32 * g;
        const int otw0 = P.brow[imin(b_w0, P.B - 1)];
        const int otw1 = P.brow[imin(b_w0 + 31, P.B - 1)];
        const int nrw = otw1 - otw0 + 1;
        const int ot = bvalid ? P.brow[b] - otw0 : 0;
        const int orow0 = otw0 - cur.ot0;
        const int myrow = bvalid ? P.brow[b] - cur.ot0 : 0;
        const int apq = bvalid ? P.bapq[b] : 0;
        const int s_y = P.fp.s_y, M = P.fp.M;
        const int wseg = a.wseg_max;
        const int pos_max = 32 * wseg - 33;
        const int pbase = cur.pbase;
        const int F2a = cur.F2a, F2b = cur.F2a + 62, F2ref = cur.F2a + 30;
        const FixedPoint fpl = P.fp;
        unsigned kb_item = 0;   // K-blocks of this item so far (the first one overwrites D)
        for (int ch = 0; ch < cur.nchunks && !abort; ++ch, ++gch) {
            const int buf = gch & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[buf], (gch >> 1) & 1, a.wait_polls))) {
                tc_timeout(a, ts, lane, &abort);
                break;
            }
            const int32_t* vnr = reinterpret_cast<const int32_t*>(smem + L.vn[buf]);
            const int32_t* cr = reinterpret_cast<const int32_t*>(smem + L.c[buf]);
            const uint32_t* pk = reinterpret_cast<const uint32_t*>(smem + L.pk[buf]);
            const float* wt = reinterpret_cast<const float*>(smem + L.w[buf]);
            // this warp's track values for its SFTs of the chunk (index e = K-block * 4 + u)
            for (int e = lane; e < per_warp; e += 32) {
                const int il = (e / TC_SLOT) * TC_KB + TC_SLOT * r + (e % TC_SLOT);
                const int vq = vnr[il];
                yp[e] = make_int2(make_Z(F2ref, vq, fpl), fp_margin(vq, fpl));
            }
            if (!DIRECT) {
                for (int e2 = lane; e2 < per_warp * nrw; e2 += 32) {
                    const int rr = e2 / per_warp, e = e2 - rr * per_warp;
                    const int il = (e / TC_SLOT) * TC_KB + TC_SLOT * r + (e % TC_SLOT);
                    const int cq = cr[(orow0 + rr) * c_stride(I) + il];
                    cp[e * wrows + rr] = make_C(F2ref, cq, fpl);
                    cpe[e * wrows + rr] = make_int2(make_C(F2a, cq, fpl), make_C(F2b, cq, fpl));
                }
            }
            const int32_t* myc = cr + myrow * c_stride(I);
            __syncwarp();
            const int i0 = ch * I;
            for (int kbl = 0; kbl < I / TC_KB; ++kbl, ++kbs) {
                const int kb = kbs & 1;
                // buffer kb is free once the MMAs of the K-block two back have read it
                if (kbs > 1 &&
                    !__all_sync(0xffffffffu, mbar_wait(&a_empty[kb], ((kbs - 2) >> 1) & 1, a.wait_polls))) {
                    tc_timeout(a, ts, lane, &abort);
                    break;
                }
                uint32_t mk[TC_SLOT];
                unsigned slow = 0u;
#pragma unroll
                for (int u = 0; u < TC_SLOT; ++u) {
                    const int e = kbl * TC_SLOT + u;
                    const int il = kbl * TC_KB + TC_SLOT * r + u;
                    const int2 z = yp[e];
                    const int cc = DIRECT ? make_C(F2ref, myc[il], fpl) : cp[e * wrows + ot];
                    const int v = z.x - __mulhi(apq, cc);
                    // in the staged segment by construction; the clamp only keeps the read in bounds
                    const unsigned pos = min((unsigned)(pbase + (v >> s_y)), (unsigned)pos_max);
                    mk[u] = row_window(pk + il * wseg, (int)pos);
                    slow |= (fp_fast_ref(v, z.y, s_y) ? 0u : 1u) << u;
                }
                if (__any_sync(0xffffffffu, slow != 0u)) {
                    // near a rounding boundary (rare): the two-ended test, else FP64 per template
                    unsigned sl = slow;
                    while (sl) {
                        const int u = __ffs(sl) - 1;
                        sl &= sl - 1u;
                        const int e = kbl * TC_SLOT + u;
                        const int il = kbl * TC_KB + TC_SLOT * r + u;
                        uint32_t m = 0u;
                        if (bvalid && i0 + il < P.N) {
                            const int2 ze = make_int2(make_Z(F2a, vnr[il], fpl), make_Z(F2b, vnr[il], fpl));
                            const int2 ce = DIRECT ? make_int2(make_C(F2a, myc[il], fpl),
                                                               make_C(F2b, myc[il], fpl))
                                                   : cpe[e * wrows + ot];
                            const int v0 = ze.x - __mulhi(apq, ce.x);
                            const int v1 = ze.y - __mulhi(apq, ce.y);
                            int path;
                            if (!fp_window_ends(v0, v1, pbase, pos_max, s_y, M, pk + il * wseg, &m, &path))
                                m = slow_window_exact(P, v0, v1, pbase, pos_max, pk + il * wseg, cur.s, b,
                                                      i0 + il, cur.j0, a.status);
                        }
#pragma unroll
                        for (int k = 0; k < TC_SLOT; ++k) mk[k] = (k == u) ? m : mk[k];
                    }
                }
                // A: byte p of a row pair's 32 is bit j = (p >> 2) + 8 (p & 3) of the window
                const uint32_t abase = smem_u32(smem + L.a[kb]);
#pragma unroll
                for (int u = 0; u < TC_SLOT; ++u) {
                    const uint32_t x = mk[u];
                    sts128(abase + a_off0 + 16u * u, x & 0x01010101u, (x >> 1) & 0x01010101u,
                           (x >> 2) & 0x01010101u, (x >> 3) & 0x01010101u);
                    sts128(abase + a_off1 + 16u * u, (x >> 4) & 0x01010101u, (x >> 5) & 0x01010101u,
                           (x >> 6) & 0x01010101u, (x >> 7) & 0x01010101u);
                }
                if (warp == 0) {
                    // B: digits of SFT kbl * 32 + lane's weight, its ones column, zeros past N
                    const int il = kbl * TC_KB + lane;
                    const bool in = i0 + il < P.N;
                    const float wf = in ? wt[il] : 0.f;
                    const float ws = wf * 16777216.0f;                      // x 2^24, exact
                    const bool fits = ws < 4294967040.0f;
                    if (!fits && in) set_status(a.status, ST_RANGE);
                    uint32_t wq = fits ? __float2uint_rn(ws) : 0xFFFFFFFFu;
                    uint32_t d[4];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        d[q] = e4m3_digit(wq & 15u) | (e4m3_digit((wq >> 4) & 15u) << 8) |
                               (e4m3_digit((wq >> 8) & 15u) << 16) | (e4m3_digit((wq >> 12) & 15u) << 24);
                        wq >>= 16;
                    }
                    d[2] = in ? 0x38u : 0u;                                 // column 8: ones (1.0)
                    d[3] = 0u;
                    sts128(smem_u32(smem + L.b[kb]) + (uint32_t)((lane >> 3) * B_LBO + (lane & 7) * 16), d[0],
                           d[1], d[2], d[3]);
                }
                fence_proxy_async();
                tmem_fence_before();
                __syncwarp();
                if (lane == 0) {
                    // the last warp to store this K-block issues its 16 MMAs and commits them to the
                    // buffer's barrier (accumulating onto the item's earlier K-blocks)
                    __threadfence_block();
                    const unsigned prev = atomicAdd(&a_cnt[kb], 1u);
                    if (prev == (unsigned)TC_PRODUCERS * ((kbs >> 1) + 1) - 1) {
                        __threadfence_block();
                        fence_proxy_async();
                        tmem_fence_after();
                        const uint64_t bd = smem_desc(smem_u32(smem + L.b[kb]), B_LBO, B_BYTES);
                        const uint64_t ad0 = smem_desc(smem_u32(smem + L.a[kb]), A_LBO, A_SBO);
#pragma unroll 1
                        for (int t = 0; t < TC_TILES; ++t)
                            tc_mma(tbase + 16u * t, ad0 + (uint64_t)(t * 8 * A_SBO / 16), bd,
                                   kb_item > 0 ? 1u : 0u);
                        tc_commit(&a_empty[kb]);
                    }
                }
                ++kb_item;
            }
            if (abort) break;
            // done with this staging buffer: the last producer warp to finish refills it two chunks ahead
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const unsigned prev = atomicAdd(&done[buf], 1u);
                if (prev == (unsigned)TC_PRODUCERS * ((gch >> 1) + 1) - 1) {
                    __threadfence_block();   // the previous issuer's writes of the item ring
                    ItemCtx nx;
                    int nch;
                    if (advance_chunk(a, pq, wk, ts, head, ch, 2, TC_TB, &nx, &nch))
                        issue_stage(a, maps, nx, nch, smem, L, buf, (int)gch + 2);
                }
            }
        }
        // the item's last MMAs are done (they complete in order): read out the sums
        if (!abort && kbs > 0 &&
            !__all_sync(0xffffffffu, mbar_wait(&a_empty[(kbs - 1) & 1], ((kbs - 1) >> 1) & 1, a.wait_polls)))
            tc_timeout(a, ts, lane, &abort);
        if (__syncthreads_or(ts.abort)) break;
        tmem_fence_after();
        tc_emit(a, P, cur, tbase, visit, ts, sm);
        tmem_fence_before();

        // the last chunk's issuer has taken the next item or found the pool exhausted
        ++head;
        if (head >= ts.q_tail) break;
        step = ts.q_step[head & 3];
        cur = item_ctx(a, decode_item(a, walk_item(wk, step)), TC_TB);
        __syncthreads();
    }
    if (!ts.abort && !a.dense && open_run >= 0) topk_close_visit<TC_THREADS>(a, visit, ts, sm);
    if (ts.abort && tid == 0) {
        // copies and MMAs still in flight into this CTA's shared and tensor memory: wait for them
        const int* inflight = inflight_slots(smem, L);
        for (int bb = 0; bb < 2; ++bb)
            if (inflight[bb] >= 0) (void)mbar_wait(&bars[bb], ((unsigned)inflight[bb] >> 1) & 1u, a.wait_polls);
    }
    if (ts.abort && tid == 0 && kbs > 0)   // (bounded: a K-block that was not stored by all warps never commits)
        (void)mbar_wait(&a_empty[(kbs - 1) & 1], ((kbs - 1) >> 1) & 1, a.wait_polls);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_free(*tslot, TC_TCOLS);
}

}  // namespace

int count_tc_smem_bytes(int I, int wseg, int ot_max, int wrows, int direct) {
    return make_tc_layout(I, wseg, ot_max, wrows, direct).total;
}

int count_tc_tile() { return TC_TB; }

void launch_count_tc(const CountArgs& a, const TmapSet& maps, int grid, cudaStream_t st) {
    // one CTA per SM: the double-buffered operands need most of its shared memory
    if (grid <= 0) return;
    if (a.direct) {
        static int s_tc1 = 0;
        ensure_smem(count_tc<true>, a.smem_bytes, &s_tc1);
        count_tc<true><<<grid, TC_THREADS, a.smem_bytes, st>>>(a, maps);
    } else {
        static int s_tc0 = 0;
        ensure_smem(count_tc<false>, a.smem_bytes, &s_tc0);
        count_tc<false><<<grid, TC_THREADS, a.smem_bytes, st>>>(a, maps);
    }
}

}  // namespace bsh

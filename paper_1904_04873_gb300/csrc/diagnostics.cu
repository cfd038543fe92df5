// Track diagnostics (Eq. (15)): per-term comparisons of the exact FP64 bin with
// the fixed-point bin used by the batched kernels and with a bin evaluated in
// single precision, and the bins of listed templates.
#include "bsh_internal.cuh"

namespace bsh {
namespace {

__device__ __forceinline__ double vn_of(const ProbDev& P, int s, int i) {
    const double* n = P.sky + 3 * (size_t)s;
    const double* v = P.v + 3 * (size_t)i;
    return __dadd_rn(__dadd_rn(__dmul_rn(v[0], n[0]), __dmul_rn(v[1], n[1])), __dmul_rn(v[2], n[2]));
}

// One thread per (s, b, i); loops over the f0 templates.
// counts: [0] terms, [1] single-precision bin != FP64 bin, [2] fixed-point bin != FP64 bin
// outside the tie band, [3] terms inside the tie band (|frac(x) - 1/2| < 1e-9).
__global__ void precision_kernel(const ProbDev* probs, int s_begin, int s_end, unsigned long long* counts) {
    const ProbDev& P = probs[0];
    const long long per = (long long)P.B * P.N;
    const long long total = (long long)(s_end - s_begin) * per;
    unsigned long long c1 = 0, c2 = 0, c3 = 0, c0 = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = s_begin + (int)(e / per);
        const long long r = e % per;
        const int b = (int)(r / P.N);
        const int i = (int)(r % P.N);
        const int ot = P.brow[b];
        const double vn = vn_of(P, s, i);
        const double c = P.c64[(size_t)ot * P.Np + i];
        const double ap = P.bap[b];
        const double D = __dsub_rn(vn, __dmul_rn(ap, c));
        // single precision evaluation of the same expression
        const float vn32 = (float)vn, c32 = (float)c, ap32 = (float)ap;
        const float D32 = __fsub_rn(vn32, __fmul_rn(ap32, c32));
        const int vq = P.vn_q[(size_t)s * P.Np + i];
        const int cq = P.c_q[(size_t)ot * P.Np + i];
        const int apq = P.bapq[b];
        const int cell = 1 << P.fp.s_y;
        for (int j = 0; j < P.n_f0; ++j) {
            const double F = P.F0 + (double)j;
            const double x = __dadd_rn(F, __dmul_rn(F, D));
            const long long k64 = (long long)floor(__dadd_rn(x, 0.5));
            const double fr = x - floor(x);
            const bool tie = fabs(fr - 0.5) < 1e-9;
            const float F32 = (float)F;
            const float x32 = __fadd_rn(F32, __fmul_rn(F32, D32));
            const long long k32 = (long long)floorf(__fadd_rn(x32, 0.5f));
            const int F2 = (int)llrint(2.0 * F);
            const int v = make_Z(F2, vq, P.fp) - mulhi32(apq, make_C(F2, cq, P.fp));
            const int frq = v & (cell - 1);
            long long kfp;
            if (frq < P.fp.M || frq > cell - P.fp.M) kfp = k64;          // the kernels' exact fallback
            else kfp = (long long)(P.G0 + j) + (long long)(v >> P.fp.s_y);
            ++c0;
            c1 += (k32 != k64);
            c2 += (!tie && kfp != k64);
            c3 += tie;
        }
    }
    atomicAdd(&counts[0], c0);
    atomicAdd(&counts[1], c1);
    atomicAdd(&counts[2], c2);
    atomicAdd(&counts[3], c3);
}

// One warp per listed template; lanes over SFTs: bins[e][i] = exact bin number.
__global__ void bins_kernel(const ProbDev* probs, const int64_t* ids, int n, int32_t* bins, unsigned* status) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n) return;
    const ProbDev& P = probs[0];
    const long long id = ids[e];
    const long long per_s = (long long)P.B * P.n_f0;
    if (id < 0 || id >= per_s * P.S) {
        if (lane == 0) set_status(status, ST_ARG);
        return;
    }
    const int s = (int)(id / per_s);
    const long long rem = id % per_s;
    const int b = (int)(rem / P.n_f0);
    const int j = (int)(rem % P.n_f0);
    const int ot = P.brow[b];
    const double ap = P.bap[b];
    const double F = P.F0 + (double)j;
    for (int i = lane; i < P.N; i += 32) {
        const double D = __dsub_rn(vn_of(P, s, i), __dmul_rn(ap, P.c64[(size_t)ot * P.Np + i]));
        const double x = __dadd_rn(F, __dmul_rn(F, D));
        bins[(size_t)e * P.N + i] = (int32_t)floor(__dadd_rn(x, 0.5));
    }
}

}  // namespace

void launch_precision(const ProbDev* dprob, int s_begin, int s_end, unsigned long long* counts, cudaStream_t st) {
    precision_kernel<<<152 * 8, 256, 0, st>>>(dprob, s_begin, s_end, counts);
}

void launch_bins(const ProbDev* dprob, const int64_t* ids, int n, int32_t* bins, unsigned* status, cudaStream_t st) {
    if (n <= 0) return;
    bins_kernel<<<(n + 7) / 8, 256, 0, st>>>(dprob, ids, n, bins, status);
}

}  // namespace bsh

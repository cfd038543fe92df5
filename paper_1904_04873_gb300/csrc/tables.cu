// Track tables (Eq. (15)): the FP64 pieces of the Doppler / binary track that
// do not depend on f0, evaluated once per call.
//   vn_q[s][i]  = round(vn * 2^s_vn),  vn = (v_x n_x + v_y n_y) + v_z n_z
//   c64[ot][i]  = Omega g,  g = (cos(phi) + kappa cos(2 phi)) + eta sin(2 phi),
//                 phi = Omega (t_i - t_asc)  (Eq. (14); g = cos(phi) when kappa = eta = 0)
//   c_q = round(c64 * 2^s_c)
// for every orbit row ot = (Omega, t_asc, kappa, eta).
//   w32 / w64   = the problem's weights widened exactly (fp16/bf16/fp32 -> fp32, any -> fp64)
// The products are rounded individually (no fused multiply-add) so that the
// FP64 values equal those of a plain sequential evaluation of the formula.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bsh_internal.cuh"

namespace bsh {
namespace {

__device__ __forceinline__ double load_weight(const void* w, int dtype, size_t idx) {
    switch (dtype) {
        case BSH_F32: return (double)static_cast<const float*>(w)[idx];
        case BSH_F16: return (double)__half2float(static_cast<const __half*>(w)[idx]);
        case BSH_BF16: return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(w)[idx]);
        default: return static_cast<const double*>(w)[idx];
    }
}

__global__ void sky_tables(const ProbDev* __restrict__ probs, int q, int mode, unsigned* status) {
    const ProbDev& P = probs[q];
    const long long total = (long long)P.S * P.Np;
    const double scale = ldexp(1.0, P.fp.s_vn);
    const double lim = 2147483000.0;
    const double vlim = P.v_max * (1.0 + 1e-12);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / P.Np), i = (int)(e % P.Np);
        int32_t vq = 0;
        double wv = 0.0;
        if (i < P.N) {
            const double* n = P.sky + 3 * (size_t)s;
            const double* v = P.v + 3 * (size_t)i;
            const double vn = __dadd_rn(__dadd_rn(__dmul_rn(v[0], n[0]), __dmul_rn(v[1], n[1])),
                                        __dmul_rn(v[2], n[2]));
            const double x = __dmul_rn(vn, scale);
            if (!(fabs(x) < lim) || !(fabs(vn) <= vlim)) set_status(status, ST_RANGE);
            else vq = __double2int_rn(x);
            wv = load_weight(P.w, P.w_dtype, (size_t)s * P.N + i);
        }
        P.vn_q[e] = vq;
        if (mode == BSH_MODE_PLAIN) P.w64[e] = wv;
        else P.w32[e] = (float)wv;   // exact for fp16 / bf16 / fp32 weights
    }
}

__global__ void binary_tables(const ProbDev* __restrict__ probs, int q, unsigned* status) {
    const ProbDev& P = probs[q];
    const long long total = (long long)P.nOT * P.Np;
    const double scale = ldexp(1.0, P.fp.s_c);
    const double lim = 2147483000.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ot = (int)(e / P.Np), i = (int)(e % P.Np);
        double c = 0.0;
        int32_t cq = 0;
        if (i < P.N) {
            const double* o = P.orb + 4 * (size_t)ot;
            const double Om = o[0], Ta = o[1], kap = o[2], eta = o[3];
            const double arg = __dmul_rn(Om, __dsub_rn(P.t[i], Ta));
            double g = cos(arg);
            if (kap != 0.0 || eta != 0.0) {
                const double a2 = __dmul_rn(2.0, arg);
                g = __dadd_rn(__dadd_rn(g, __dmul_rn(kap, cos(a2))), __dmul_rn(eta, sin(a2)));
            }
            c = __dmul_rn(Om, g);
            const double x = __dmul_rn(c, scale);
            if (!(fabs(x) < lim)) set_status(status, ST_RANGE);
            else cq = __double2int_rn(x);
        }
        P.c64[e] = c;
        P.c_q[e] = cq;
    }
}

}  // namespace

void launch_tables(const ProbDev& hp, const ProbDev* dprob, int mode, unsigned* status, cudaStream_t st) {
    // hp is the host copy of the device descriptor at index q; its q is stored in region_base order,
    // so the caller passes dprob already offset to the problem.
    const int threads = 256;
    long long n1 = (long long)hp.S * hp.Np;
    long long b1 = (n1 + threads - 1) / threads;
    if (b1 > 65536) b1 = 65536;
    if (b1 > 0) sky_tables<<<(unsigned)b1, threads, 0, st>>>(dprob, 0, mode, status);
    long long n2 = (long long)hp.nOT * hp.Np;
    long long b2 = (n2 + threads - 1) / threads;
    if (b2 > 65536) b2 = 65536;
    if (b2 > 0) binary_tables<<<(unsigned)b2, threads, 0, st>>>(dprob, 0, status);
}

}  // namespace bsh

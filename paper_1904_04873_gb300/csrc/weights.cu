// Weights (Sec. IV.A, Eq. (22)): w_i(n) = (F+^2 + Fx^2)(n, t_i) / S_n,i, scaled
// per sky point to sum to N, rounded to the stored dtype.
//
// F+^2 + Fx^2 is computed without a polarisation basis: for the detector
// tensor D = (u u^T - v v^T)/2 and the transverse projector P = I - n n^T,
// the transverse-traceless part D_TT = P D P - P tr(P D)/2 satisfies
// F+^2 + Fx^2 = 2 D_TT : D_TT = 2 (D:D - 2 |D n|^2 + (n.D n)^2) - (tr D - n.D n)^2.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bsh_internal.cuh"

namespace bsh {
namespace {

__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ double antenna_f2(const double* n, const double* arm) {
    const double* u = arm;
    const double* v = arm + 3;
    const double un = dot3(u, n), vn = dot3(v, n);
    const double uu = dot3(u, u), vv = dot3(v, v), uv = dot3(u, v);
    const double DD = 0.25 * (uu * uu + vv * vv - 2.0 * uv * uv);
    const double Dn2 = 0.25 * (un * un * uu + vn * vn * vv - 2.0 * un * vn * uv);
    const double alpha = 0.5 * (un * un - vn * vn);
    const double tau = 0.5 * (uu - vv);
    const double ta = tau - alpha;
    return 2.0 * (DD - 2.0 * Dn2 + alpha * alpha) - ta * ta;
}

template <int THREADS>
__device__ double block_sum(double x, double* s_red) {
    // fixed tree: deterministic for a given launch shape
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_red[warp] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < THREADS / 32; ++w) r += s_red[w];
        s_red[THREADS / 32] = r;
    }
    __syncthreads();
    return s_red[THREADS / 32];
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) weights_kernel(const double* __restrict__ sky, const double* __restrict__ arms,
                                                          const double* __restrict__ Sn, int N, int norm, int dtype,
                                                          void* __restrict__ w, double* __restrict__ sum_w,
                                                          double* __restrict__ sum_w2, unsigned* status) {
    __shared__ double s_red[THREADS / 32 + 1];
    const int s = blockIdx.x;
    double n[3] = {sky[3 * (size_t)s], sky[3 * (size_t)s + 1], sky[3 * (size_t)s + 2]};
    double part = 0.0;
    for (int i = threadIdx.x; i < N; i += THREADS) part += antenna_f2(n, arms + 6 * (size_t)i) / Sn[i];
    const double tot = block_sum<THREADS>(part, s_red);
    double scale = 1.0;
    if (norm) {
        if (!(tot > 0.0)) {
            if (threadIdx.x == 0) set_status(status, ST_RANGE);
            scale = 0.0;
        } else {
            scale = __ddiv_rn((double)N, tot);
        }
    }
    double q1 = 0.0, q2 = 0.0;
    for (int i = threadIdx.x; i < N; i += THREADS) {
        const double raw = antenna_f2(n, arms + 6 * (size_t)i) / Sn[i];
        const double x = norm ? __dmul_rn(raw, scale) : raw;
        double q;
        const size_t idx = (size_t)s * N + i;
        switch (dtype) {
            case BSH_F32: {
                const float f = __double2float_rn(x);
                static_cast<float*>(w)[idx] = f;
                q = (double)f;
            } break;
            case BSH_F16: {
                const __half h = __double2half(x);
                static_cast<__half*>(w)[idx] = h;
                q = (double)__half2float(h);
            } break;
            case BSH_BF16: {
                const __nv_bfloat16 h = __double2bfloat16(x);
                static_cast<__nv_bfloat16*>(w)[idx] = h;
                q = (double)__bfloat162float(h);
            } break;
            default:
                static_cast<double*>(w)[idx] = x;
                q = x;
        }
        q1 += q;
        q2 += q * q;
    }
    const double t1 = block_sum<THREADS>(q1, s_red);
    const double t2 = block_sum<THREADS>(q2, s_red);
    if (threadIdx.x == 0) {
        if (sum_w) sum_w[s] = t1;
        if (sum_w2) sum_w2[s] = t2;
    }
}

}  // namespace

int launch_weights(const double* sky, int S, const double* arms, const double* Sn, int N, int norm,
                   int dtype, void* w, double* sum_w, double* sum_w2, unsigned* status, cudaStream_t st) {
    if (S <= 0) return 0;
    weights_kernel<256><<<S, 256, 0, st>>>(sky, arms, Sn, N, norm, dtype, w, sum_w, sum_w2, status);
    return 0;
}

}  // namespace bsh

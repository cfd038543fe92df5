// Weights (Sec. IV.A, Eq. (22)): w_i(n) = (F+^2 + Fx^2)(n, t_i) / S_n,i, scaled
// per sky point to sum to N, rounded to the stored dtype.
//
// F+ and Fx are the contractions of the detector tensor D = (u u^T - v v^T)/2
// (arm unit vectors u, v at the SFT mid-time) with the polarisation tensors
// e+ = p p^T - q q^T and ex = p q^T + q p^T of the wave frame (Eq. (1)):
//   F+ = ((u.p)^2 - (u.q)^2 - ((v.p)^2 - (v.q)^2)) / 2,  Fx = (u.p)(u.q) - (v.p)(v.q),
// with p = e_alpha, q = e_delta: e_alpha = z x n / |z x n| (east on the sky), e_delta =
// n x e_alpha, at polarisation angle 0 (F+^2 + Fx^2 does not depend on it).  Every
// FP64 operation is rounded on its own (no fused multiply-add) and the normalisation
// sum runs over the SFTs in ascending order, one rounding per addition, so that the
// weights are the correctly rounded values of this definition, evaluated in a fixed
// order: every caller who follows the same order gets the same bits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bsh_internal.cuh"

namespace bsh {
namespace {

constexpr int WT = 256;         // threads per CTA (one CTA per sky point)
constexpr int TILE = 4096;      // raw weights staged per pass of the sequential sum

__device__ __forceinline__ double dot3_rn(const double* a, const double* b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// Wave-frame basis of direction n: p = e_alpha, q = e_delta (polarisation angle 0).
struct Basis {
    double p[3], q[3];
};

__device__ __forceinline__ Basis wave_basis(const double* n) {
    const double nx = n[0], ny = n[1], nz = n[2];
    const double rxy = __dsqrt_rn(__dadd_rn(__dmul_rn(nx, nx), __dmul_rn(ny, ny)));
    double ea[3];
    if (rxy > 1e-300) {
        ea[0] = __ddiv_rn(-ny, rxy);
        ea[1] = __ddiv_rn(nx, rxy);
        ea[2] = 0.0;
    } else {      // n along the z axis: any transverse pair serves
        ea[0] = 0.0;
        ea[1] = 1.0;
        ea[2] = 0.0;
    }
    double ed[3];
    ed[0] = __dsub_rn(__dmul_rn(ny, ea[2]), __dmul_rn(nz, ea[1]));
    ed[1] = __dsub_rn(__dmul_rn(nz, ea[0]), __dmul_rn(nx, ea[2]));
    ed[2] = __dsub_rn(__dmul_rn(nx, ea[1]), __dmul_rn(ny, ea[0]));
    // rotation by the polarisation angle psi = 0: cos = 1, sin = 0 (kept as products so that
    // the signs of zero components come out as the rotation gives them)
    const double cp = 1.0, sp = 0.0;
    Basis B;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        B.p[k] = __dadd_rn(__dmul_rn(cp, ea[k]), __dmul_rn(sp, ed[k]));
        B.q[k] = __dadd_rn(__dmul_rn(-sp, ea[k]), __dmul_rn(cp, ed[k]));
    }
    return B;
}

// (F+^2 + Fx^2) / S_n for arms u = arm[0..2], v = arm[3..5].
__device__ __forceinline__ double raw_weight(const Basis& B, const double* arm, double Sn) {
    const double* u = arm;
    const double* v = arm + 3;
    const double up = dot3_rn(u, B.p), uq = dot3_rn(u, B.q), vp = dot3_rn(v, B.p), vq = dot3_rn(v, B.q);
    const double Fp = __dmul_rn(0.5, __dsub_rn(__dsub_rn(__dmul_rn(up, up), __dmul_rn(uq, uq)),
                                               __dsub_rn(__dmul_rn(vp, vp), __dmul_rn(vq, vq))));
    const double Fc = __dsub_rn(__dmul_rn(up, uq), __dmul_rn(vp, vq));
    return __ddiv_rn(__dadd_rn(__dmul_rn(Fp, Fp), __dmul_rn(Fc, Fc)), Sn);
}

__device__ double block_sum(double x, double* s_red) {
    // fixed tree: deterministic for a given launch shape (used for the sums of the stored
    // weights, which only feed the significance of Eq. (25))
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_red[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < WT / 32; ++w) r += s_red[w];
        s_red[WT / 32] = r;
    }
    __syncthreads();
    return s_red[WT / 32];
}

__global__ void __launch_bounds__(WT) weights_kernel(const double* __restrict__ sky, const double* __restrict__ arms,
                                                     const double* __restrict__ Sn, int N, int norm, int dtype,
                                                     void* __restrict__ w, double* __restrict__ sum_w,
                                                     double* __restrict__ sum_w2, unsigned* status) {
    __shared__ double s_raw[TILE];
    __shared__ double s_red[WT / 32 + 1];
    __shared__ double s_scale;
    const int s = blockIdx.x;
    const double n[3] = {sky[3 * (size_t)s], sky[3 * (size_t)s + 1], sky[3 * (size_t)s + 2]};
    const Basis B = wave_basis(n);
    double scale = 1.0;
    if (norm) {
        // sum over i ascending, one rounding per addition: tiles of raw weights are formed in
        // parallel and added by one thread
        double tot = 0.0;
        for (int i0 = 0; i0 < N; i0 += TILE) {
            const int m = N - i0 < TILE ? N - i0 : TILE;
            for (int k = threadIdx.x; k < m; k += WT) s_raw[k] = raw_weight(B, arms + 6 * (size_t)(i0 + k), Sn[i0 + k]);
            __syncthreads();
            if (threadIdx.x == 0)
                for (int k = 0; k < m; ++k) tot = __dadd_rn(tot, s_raw[k]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (!(tot > 0.0)) {
                set_status(status, ST_RANGE);
                s_scale = 0.0;
            } else {
                s_scale = __ddiv_rn((double)N, tot);
            }
        }
        __syncthreads();
        scale = s_scale;
    }
    // a band of at most TILE SFTs still has its raw weights in shared memory (the FP64 pipe is
    // narrow on this GPU: forming them once saves half of the kernel's time)
    const bool staged = norm && N <= TILE;
    double q1 = 0.0, q2 = 0.0;
    for (int i = threadIdx.x; i < N; i += WT) {
        const double raw = staged ? s_raw[i] : raw_weight(B, arms + 6 * (size_t)i, Sn[i]);
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
    const double t1 = block_sum(q1, s_red);
    const double t2 = block_sum(q2, s_red);
    if (threadIdx.x == 0) {
        if (sum_w) sum_w[s] = t1;
        if (sum_w2) sum_w2[s] = t2;
    }
}

}  // namespace

int launch_weights(const double* sky, int S, const double* arms, const double* Sn, int N, int norm,
                   int dtype, void* w, double* sum_w, double* sum_w2, unsigned* status, cudaStream_t st) {
    if (S <= 0) return 0;
    weights_kernel<<<S, WT, 0, st>>>(sky, arms, Sn, N, norm, dtype, w, sum_w, sum_w2, status);
    return 0;
}

}  // namespace bsh

// Binary template bank with the spacings of Eq. (30)-(32) (Sec. V.B), host code.
//
// The resolutions depend on where in the binary parameter space they are evaluated
// (delta a_p ~ 1/Omega, delta Omega ~ 1/(a_p Omega), delta t_asc ~ 1/(a_p Omega^2)), so
// the bank is not a Cartesian grid.  It is laid out as orbit rows (Omega, t_asc) that
// each carry a block of a_p values, the layout the count kernels stage:
//   - Omega from 2 pi / P_max upwards, each step the spacing at the largest a_p of the
//     range (the smallest delta Omega at that Omega), until past 2 pi / P_min;
//   - at each Omega, a_p from a_min upwards in steps of delta a_p(Omega) up to a_max;
//   - the a_p values are cut into blocks whose largest / smallest ratio is at most
//     ap_block, and each block gets its own t_asc grid, spaced by delta t_asc at the
//     block's largest a_p, over one period around t_mid (Eq. (35)).
// Every step is taken at the point where the spacing is smallest, so the bank is
// never coarser than the metric asks for anywhere.
#include <cmath>
#include <cstdint>
#include <vector>

#include "bsh_internal.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;

void resolution(double f, double T_c, double T_obs, double a_p, double Om, double m_a, double m_Om, double m_t,
                double* d_ap, double* d_Om, double* d_t) {
    *d_ap = std::sqrt(6.0 * m_a) / (PI * T_c * f * Om);
    *d_Om = std::sqrt(72.0 * m_Om) / (PI * T_c * f * a_p * Om * T_obs);
    *d_t = std::sqrt(6.0 * m_t) / (PI * T_c * f * a_p * Om * Om);
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" int bsh_binary_resolution(double f, double T_c, double T_obs, double a_p, double Omega, double m_a,
                                     double m_Om, double m_t, double* d_ap, double* d_Om, double* d_t) {
    if (!d_ap || !d_Om || !d_t) return BSH_ERR_ARG;
    if (!finite_pos(f) || !finite_pos(T_c) || !finite_pos(T_obs) || !finite_pos(a_p) || !finite_pos(Omega) ||
        !finite_pos(m_a) || !finite_pos(m_Om) || !finite_pos(m_t))
        return BSH_ERR_ARG;
    resolution(f, T_c, T_obs, a_p, Omega, m_a, m_Om, m_t, d_ap, d_Om, d_t);
    return BSH_OK;
}

extern "C" int bsh_template_bank(const bsh_bank_spec* spec, int* n_orbit, double* orbit, int orbit_cap, int* n_bank,
                                 int32_t* bank_orbit, double* bank_ap, int bank_cap) {
    if (!spec || !n_orbit || !n_bank) return BSH_ERR_ARG;
    const bsh_bank_spec& q = *spec;
    if (!finite_pos(q.f) || !finite_pos(q.T_c) || !finite_pos(q.T_obs) || !std::isfinite(q.t_mid) ||
        !finite_pos(q.ap_min) || !(q.ap_max >= q.ap_min) || !std::isfinite(q.ap_max) || !finite_pos(q.P_min) ||
        !(q.P_max >= q.P_min) || !std::isfinite(q.P_max) || !finite_pos(q.m_a) || !finite_pos(q.m_Om) ||
        !finite_pos(q.m_t) || !(q.ap_block >= 1.0) || !std::isfinite(q.ap_block))
        return BSH_ERR_ARG;
    if (!(q.P_min > q.T_c)) return BSH_ERR_RANGE;   // the spacings assume T_c << P
    const double Om_lo = 2.0 * PI / q.P_max, Om_hi = 2.0 * PI / q.P_min;
    const long long limit = 1LL << 30;
    long long rows = 0, tmpl = 0;
    std::vector<double> aps;
    double Om = Om_lo;
    while (true) {
        double d_ap, d_Om, d_t;
        resolution(q.f, q.T_c, q.T_obs, q.ap_max, Om, q.m_a, q.m_Om, q.m_t, &d_ap, &d_Om, &d_t);
        aps.clear();
        for (long long k = 0;; ++k) {
            const double a = q.ap_min + (double)k * d_ap;
            if (a > q.ap_max) break;
            aps.push_back(a);
            if ((long long)aps.size() > limit) return BSH_ERR_RANGE;
        }
        const double P = 2.0 * PI / Om;
        size_t i0 = 0;
        while (i0 < aps.size()) {
            size_t i1 = i0 + 1;
            while (i1 < aps.size() && aps[i1] <= q.ap_block * aps[i0]) ++i1;
            double dA, dO, dT;
            resolution(q.f, q.T_c, q.T_obs, aps[i1 - 1], Om, q.m_a, q.m_Om, q.m_t, &dA, &dO, &dT);
            for (long long k = 0;; ++k) {
                const double t = (q.t_mid - 0.5 * P) + (double)k * dT;
                if (!(t < q.t_mid + 0.5 * P)) break;
                if (rows >= limit || tmpl + (long long)(i1 - i0) > limit) return BSH_ERR_RANGE;
                if (orbit && rows < orbit_cap) {
                    orbit[4 * rows] = Om;
                    orbit[4 * rows + 1] = t;
                    orbit[4 * rows + 2] = 0.0;
                    orbit[4 * rows + 3] = 0.0;
                }
                for (size_t i = i0; i < i1; ++i) {
                    if (bank_orbit && bank_ap && tmpl < bank_cap) {
                        bank_orbit[tmpl] = (int32_t)rows;
                        bank_ap[tmpl] = aps[i];
                    }
                    ++tmpl;
                }
                ++rows;
            }
            i0 = i1;
        }
        Om += d_Om;
        if (Om > Om_hi) break;
    }
    *n_orbit = (int)rows;
    *n_bank = (int)tmpl;
    if ((orbit && rows > orbit_cap) || ((bank_orbit || bank_ap) && tmpl > bank_cap)) return BSH_ERR_WORKSPACE;
    return BSH_OK;
}

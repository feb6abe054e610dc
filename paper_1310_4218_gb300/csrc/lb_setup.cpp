// Host-side set-up shared by every entry point that launches the step
// kernel (lb_create and lb_step_noalloc): per-grid argument checks, the
// zero-flux pivots, the kernel choice and the device record of a grid.
// One copy, so the two entry points cannot drift apart.
#include <cmath>
#include <cstring>

#include "lb_internal.h"

namespace lbk {

const char *check_grid_desc(const lb_grid_desc &d) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nz > kNzMax)
        return "need nx, ny >= 1 and 1 <= nz <= 128";
    if ((long long)d.nx * d.ny * d.nz >= (1LL << 31)) return "nx*ny*nz must be below 2^31";
    if (d.dynamics != 0 && d.dynamics != 1) return "dynamics is 0 (advection) or 1 (Jacobi)";
    if (d.pitch != 0 && d.pitch < d.nx) return "pitch must be 0 or at least nx";
    if ((long long)(d.pitch ? d.pitch : d.nx) * d.ny * d.nz >= (1LL << 31))
        return "pitch*ny*nz must be below 2^31";
    if (d.dynamics == 0 &&
        (!std::isfinite(d.cx) || !std::isfinite(d.cy) || !std::isfinite(d.cz) ||
         std::fabs(d.cx) + std::fabs(d.cy) + std::fabs(d.cz) > 1.0 + 1e-12))
        return "need |cx|+|cy|+|cz| <= 1";
    if (d.dynamics == 1 && !(d.nu > 0.0 && d.nu <= 1.0 / 6.0 + 1e-15))
        return "Jacobi weight needs 0 < nu <= 1/6";
    if (!std::isfinite(d.r) || d.r < 0.0) return "need r >= 0";
    const bool ok_types = (d.storage == LB_F64 && d.compute == LB_F64) ||
                          (d.storage == LB_F64 && d.compute == LB_F32) ||
                          (d.storage == LB_F32 && d.compute == LB_F32) ||
                          (d.storage == LB_BF16 && d.compute == LB_F32);
    if (!ok_types) return "unsupported storage/compute pair";
    if (!d.q0 || !d.q1 || d.q0 == d.q1) return "q0 and q1 must be distinct device buffers";
    if (d.kc_disk != 0 && d.kc_disk != 1) return "kc_disk is 0 or 1";
    if (!d.kc_disk && !d.kc) return "kc array required";
    if (d.kc_disk && (d.k_in < 0 || d.k_out < 0 || d.disk_r < 0))
        return "disk needs k_in, k_out, R >= 0";
    if (d.kc_disk && (d.k_in > LB_KC_MAX || d.k_out > LB_KC_MAX))
        return "disk needs k_in, k_out <= LB_KC_MAX";
    if (d.compute == LB_F64 && d.nz > 64) return "FP64 compute supports nz <= 64";
    return nullptr;
}

// M = tridiag(-r, 1+2r, -r) with first and last diagonal 1+r; forward
// elimination pivots m_k = 1 / (b_k - r^2 m_{k-1}).
void zero_flux_pivots(double r, int exact_nz, double *m) {
    for (int k = 0; k < kNzMax; ++k) {
        if (exact_nz > 0 && k >= exact_nz) {
            m[k] = 1.0;
            continue;
        }
        const bool last = exact_nz > 0 && k == exact_nz - 1;
        const int nb = (k > 0 ? 1 : 0) + (last ? 0 : 1);   // neighbours of row k
        const double b = 1.0 + r * nb;
        m[k] = k == 0 ? 1.0 / b : 1.0 / (b - r * r * m[k - 1]);
    }
}

double zero_flux_last_pivot(double r, int nz) {
    if (nz == 1) return 1.0;
    double m = 1.0 / (1.0 + r);
    for (int k = 1; k < nz - 1; ++k) m = 1.0 / (1.0 + 2.0 * r - r * r * m);
    return 1.0 / (1.0 + r - r * r * m);
}

double converged_pivot(double r) {
    // fixed point of m = 1 / (1 + 2r - r^2 m), a contraction (factor (r m)^2 < 1)
    double m = 1.0 / (1.0 + r);
    for (int it = 0; it < 4000; ++it) {
        const double n = 1.0 / (1.0 + 2.0 * r - r * r * m);
        if (n == m) break;
        m = n;
    }
    return m;
}

bool twin_pivots_converge(double r) {
    double mt[kNzMax];
    zero_flux_pivots(r, 0, mt);
    const double minf = converged_pivot(r);
    for (int k = kTwinS0; k < kNzMax / 2; ++k)
        if ((float)(mt[k] / minf) != 1.0f || (float)(r * mt[k]) != (float)(r * mt[kTwinS0]))
            return false;
    return true;
}

bool layout_is_wide(const lb_vp *vps, int nvps, bool any_jacobi) {
    long long cols_all = 0, cols_wide = 0;
    for (int v = 0; v < nvps; ++v) {
        const long long c = (long long)vps[v].w * vps[v].h;
        cols_all += c;
        if (vps[v].w % 16 == 0) cols_wide += c;
    }
    return 4 * cols_wide >= 3 * cols_all || any_jacobi;
}

bool choose_step_kernel(const lb_grid_desc *grids, int ngrids, const lb_vp *vps, int nvps,
                        int threads_hint, bool staged, KernelInfo *out, int ctas_per_sm) {
    int nzmax = 0, nzmin = kNzMax;
    bool any_jacobi = false;
    for (int g = 0; g < ngrids; ++g) {
        nzmax = grids[g].nz > nzmax ? grids[g].nz : nzmax;
        nzmin = grids[g].nz < nzmin ? grids[g].nz : nzmin;
        any_jacobi = any_jacobi || grids[g].dynamics == 1;
    }
    return find_step_kernel(grids[0].storage, grids[0].compute, nzmax, nzmin, nzmax == nzmin, out,
                            threads_hint, staged, layout_is_wide(vps, nvps, any_jacobi),
                            twin_pivots_converge(grids[0].r), ctas_per_sm);
}

template <class TC>
static void fill_coef_t(double r, const KernelInfo &k, Coef<TC> &c) {
    double m[kNzMax];
    // split and twin kernels eliminate from both ends: the pivots of a
    // column that starts at a zero-flux end, and the middle 2x2 coupling
    pivots_for_kernel(r, k, m);
    for (int i = 0; i < kNzMax; ++i) {
        c.m[i] = (TC)m[i];
        c.rm[i] = (TC)(r * m[i]);
    }
    const double a = k.split ? r * m[k.nz_variant / 2 - 1] : 0.0;
    c.ifa = (TC)a;
    c.ifc = (TC)(1.0 / (1.0 - a * a));
    // scaled solves of the split family (the length-independent table)
    const double minf = converged_pivot(r);
    for (int i = 0; i < kNzMax; ++i) c.e[i] = (TC)(m[i] / minf);
    for (int i = 0; i < kTwinS0; ++i) {
        const float e = (float)(m[i] / minf), rm = (float)(r * m[i]);
        c.e2[i] = {e, e};
        c.rm2[i] = {rm, rm};
    }
    // a solve grows a column by at most 1 / m_inf (M^-1 has unit row sums
    // and nonnegative entries): rescale before the growth reaches 2^40
    const double g = -std::log2(minf);
    int every = g > 0.0 ? (int)std::floor(40.0 / g) : 16;
    every = every < 1 ? 1 : (every > 16 ? 16 : every);
    const double resc = std::pow(minf, every);
    c.resc = (TC)resc;
    c.resc_every = every;
    const double lr = std::log((double)c.resc), lm = std::log(minf);
    for (int kk = 0; kk <= LB_KC_MAX; ++kk)
        c.f[kk] = (TC)std::exp(kk * lm - (kk / every) * lr);
}

void pivots_for_kernel(double r, const KernelInfo &k, double *m) {
    zero_flux_pivots(r, (k.exact && !k.split) ? k.nz_variant : 0, m);
}

void fill_coef(double r, const KernelInfo &k, Coef<float> &c) { fill_coef_t(r, k, c); }
void fill_coef(double r, const KernelInfo &k, Coef<double> &c) { fill_coef_t(r, k, c); }

void fill_grid_dev(const lb_grid_desc &d, int32_t *kc_range, GridDev &h) {
    std::memset(&h, 0, sizeof(h));
    h.nx = d.nx;
    h.ny = d.ny;
    h.nz = d.nz;
    h.kc_disk = d.kc_disk;
    h.pitch = d.pitch ? d.pitch : d.nx;
    h.plane = h.pitch * d.ny;
    h.sx = d.cx >= 0 ? 1 : -1;
    h.sy = d.cy >= 0 ? 1 : -1;
    h.sz = d.cz >= 0 ? 1 : -1;
    h.q[0] = d.q0;
    h.q[1] = d.q1;
    h.kc = d.kc;
    h.kc_range = kc_range;
    h.disk_x0 = d.disk_x0;
    h.disk_y0 = d.disk_y0;
    h.disk_vx = d.disk_vx;
    h.disk_vy = d.disk_vy;
    h.disk_r = d.disk_r;
    h.k_in = d.k_in;
    h.k_out = d.k_out;
    const double w[4] = {1.0 - std::fabs(d.cx) - std::fabs(d.cy) - std::fabs(d.cz),
                         std::fabs(d.cx), std::fabs(d.cy), std::fabs(d.cz)};
    for (int n = 0; n < 4; ++n) {
        h.wd[n] = w[n];
        h.wf[n] = (float)w[n];
    }
    h.xy_only = (d.dynamics == 0 && w[0] == 0.0 && d.cz == 0.0) ? 1 : 0;
    h.jacobi = d.dynamics == 1 ? 1 : 0;
    h.nu_d = d.nu;
    h.w0j_d = 1.0 - 6.0 * d.nu;
    h.nu_f = (float)d.nu;
    h.w0j_f = (float)(1.0 - 6.0 * d.nu);
    h.sweeps_on = d.r > 0.0 ? 1 : 0;
    const double ml = zero_flux_last_pivot(d.r, d.nz);
    h.mlast_d = ml;
    h.rlast_d = d.r * ml;
    h.mlast_f = (float)ml;
    h.rlast_f = (float)(d.r * ml);
    if (d.nz >= 2) split_coupling(d.r, d.nz, &h.ifa_b_f, &h.ifa_t_f, &h.ifc_bt_f);
}

}  // namespace lbk

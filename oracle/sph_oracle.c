/*
 * sph_oracle.c -- plain FP64 brute-force SPH, used ONLY as test infrastructure.
 *
 * This file is the oracle that the GPU path is checked against.  It is not
 * part of the product: only tests/, the smoke check in __graft_entry__.py and
 * the CPU-baseline leg of bench.py load it.  It shares no code, header or
 * constant with the CUDA library; every formula below is written out from
 * the paper (arXiv:2511.11425, "SPH in pkdgrav3 I"), section by section:
 *
 *   kernels            Sec. 2.3 (cubic spline, Wendland C2/C4/C6 are named but
 *                      not printed; the textbook 3D forms with compact support
 *                      radius h are used, W(r,h) = w(r/h)/h^3)
 *   density + h        Sec. 2.3.3, Eq. (Density_estimate), the constant-mass
 *                      criterion M = 4/3 pi R^3(h) rho with Newton-Raphson on h,
 *                      and the grad-h term Omega
 *   EOS                Sec. 2.3.1, ideal gas P = (gamma-1) rho u
 *   forces             Sec. 2.3.5: momentum equation (gather + scatter),
 *                      PdV internal-energy equation, Monaghan viscosity
 *                      Pi_ij with mu_ij, averaged kernel for the viscous terms,
 *                      Eq. (AV_heating)
 *   time step          Sec. 2.3.6: acceleration criterion and Eq. (courant_condition)
 *
 * Every sum runs over ALL particles j (O(N^2)); there are no cells, no lists,
 * no blocking.  Periodic axes use the minimum image.  OpenMP parallelises the
 * loop over sink particles only, so every per-sink sum is in plain j order.
 */
#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <stdint.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_WC2 = 0, ORC_WC4 = 1, ORC_WC6 = 2, ORC_M4 = 3 };

typedef struct {
    int    kernel;          /* ORC_WC2 | ORC_WC4 | ORC_WC6 | ORC_M4            */
    int    max_iter;        /* Newton iterations cap                           */
    double n_ngb;           /* target 4/3 pi h^3 rho / m                       */
    double gamma;           /* ideal-gas adiabatic index                       */
    double alpha, beta;     /* Monaghan viscosity parameters                   */
    double eps_av;          /* epsilon in the mu_ij denominator                */
    double eta_courant;     /* eta_C                                           */
    double eta_acc;         /* eta_a                                           */
    double h_rel_tol;       /* Newton stop: |dh|/h < tol                       */
    double box_lo[3];
    double box_hi[3];
    int    periodic[3];
    int    pad_;
} orc_params;

/* ---- kernels: dimensionless w(q) and w'(q) for q = r/h, support q < 1 ---- */

static double kern_w(int k, double q)
{
    if (q >= 1.0) return 0.0;
    double t = 1.0 - q;
    switch (k) {
    case ORC_WC2:  /* Wendland C2: (1-q)^4 (1+4q) */
        return 21.0 / (2.0 * M_PI) * pow(t, 4) * (1.0 + 4.0 * q);
    case ORC_WC4:  /* Wendland C4: (1-q)^6 (1 + 6q + 35/3 q^2) */
        return 495.0 / (32.0 * M_PI) * pow(t, 6) * (1.0 + 6.0 * q + 35.0 / 3.0 * q * q);
    case ORC_WC6:  /* Wendland C6: (1-q)^8 (1 + 8q + 25q^2 + 32q^3) */
        return 1365.0 / (64.0 * M_PI) * pow(t, 8) *
               (1.0 + 8.0 * q + 25.0 * q * q + 32.0 * q * q * q);
    case ORC_M4:   /* cubic spline, support 1 */
        if (q < 0.5) return 8.0 / M_PI * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
        return 8.0 / M_PI * 2.0 * t * t * t;
    }
    return NAN;
}

static double kern_dw(int k, double q)
{
    if (q >= 1.0) return 0.0;
    double t = 1.0 - q;
    switch (k) {
    case ORC_WC2:  /* d/dq (1-q)^4(1+4q) = -20 q (1-q)^3 */
        return 21.0 / (2.0 * M_PI) * (-20.0 * q * pow(t, 3));
    case ORC_WC4:  /* -(56/3) q (1-q)^5 (1+5q) */
        return 495.0 / (32.0 * M_PI) * (-56.0 / 3.0 * q * pow(t, 5) * (1.0 + 5.0 * q));
    case ORC_WC6:  /* -22 q (1-q)^7 (1 + 7q + 16q^2) */
        return 1365.0 / (64.0 * M_PI) * (-22.0 * q * pow(t, 7) * (1.0 + 7.0 * q + 16.0 * q * q));
    case ORC_M4:
        if (q < 0.5) return 8.0 / M_PI * (-12.0 * q + 18.0 * q * q);
        return 8.0 / M_PI * (-6.0 * t * t);
    }
    return NAN;
}

/* W(r,h), dW/dr and dW/dh for W = w(r/h)/h^3 */
static double W_of(int k, double r, double h) { return kern_w(k, r / h) / (h * h * h); }
static double dWdr_of(int k, double r, double h) { return kern_dw(k, r / h) / (h * h * h * h); }
static double dWdh_of(int k, double r, double h)
{
    double q = r / h;
    return -(3.0 * kern_w(k, q) + q * kern_dw(k, q)) / (h * h * h * h);
}

/* r_ij = x_i - x_j with the minimum image on periodic axes */
static void separation(const orc_params *p, const double *xi, const double *xj, double d[3])
{
    for (int a = 0; a < 3; ++a) {
        d[a] = xi[a] - xj[a];
        if (p->periodic[a]) {
            double L = p->box_hi[a] - p->box_lo[a];
            d[a] -= L * nearbyint(d[a] / L);
        }
    }
}

/* threads the parallel loops use */
int orc_num_threads(void) { return omp_get_max_threads(); }

void orc_kernel_eval(int kernel, int64_t n, const double *q, double *w, double *dw)
{
    for (int64_t i = 0; i < n; ++i) {
        w[i] = kern_w(kernel, q[i]);
        dw[i] = kern_dw(kernel, q[i]);
    }
}

/* rho_i(h) = sum_j m_j W(r_ij, h) (self included) and its h-derivative;
 * also the number of j != i strictly inside h. */
static void density_sums(const orc_params *p, int64_t n, const double *pos, const double *m,
                         int64_t i, double h, double *rho, double *drho_dh, int64_t *count)
{
    double s = 0.0, ds = 0.0;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
        double d[3];
        separation(p, pos + 3 * i, pos + 3 * j, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r >= h) continue;
        s += m[j] * W_of(p->kernel, r, h);
        ds += m[j] * dWdh_of(p->kernel, r, h);
        if (j != i) ++c;
    }
    *rho = s;
    *drho_dh = ds;
    *count = c;
}

/*
 * Smoothing length and density for the listed sinks (Sec. 2.3.3).
 * Newton-Raphson on g(h) = 4/3 pi h^3 rho_i(h) - N_ngb m_i, which keeps the
 * mass inside the kernel constant; g is non-decreasing in h, so a bracket
 * [lo, hi] is kept and a step that leaves it is replaced by bisection (or by
 * doubling while no upper bound is known).  After convergence rho, Omega and
 * the neighbour count are evaluated at the final h.
 * iters_out[s] = Newton steps taken, or -1 if max_iter was reached.
 * Returns the number of sinks that did not converge.
 */
int64_t orc_density_h(const orc_params *p, int64_t n, const double *pos, const double *m,
                      int64_t ns, const int64_t *sinks, const double *h_seed,
                      double *h_out, double *rho_out, double *omega_out,
                      int64_t *nngb_out, int32_t *iters_out)
{
    int64_t failed = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : failed)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sinks ? sinks[s] : s;
        double h = h_seed[s], lo = 0.0, hi = INFINITY;
        double target = p->n_ngb * m[i];
        int it, conv = 0;
        for (it = 0; it < p->max_iter; ++it) {
            double rho, drho;
            int64_t c;
            density_sums(p, n, pos, m, i, h, &rho, &drho, &c);
            double M = 4.0 / 3.0 * M_PI * h * h * h * rho;
            double dM = 4.0 * M_PI * h * h * rho + 4.0 / 3.0 * M_PI * h * h * h * drho;
            double g = M - target;
            if (g < 0.0) lo = h; else hi = h;
            double hn = (dM > 0.0) ? h - g / dM : NAN;
            /* a Newton step below the tolerance ends the iteration (it may
             * land exactly on the bracket end that h itself just set) */
            if (isfinite(hn) && fabs(hn - h) < p->h_rel_tol * h) { h = hn; conv = 1; ++it; break; }
            if (!(hn > lo && hn < hi)) hn = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * h;
            double dh = hn - h;
            h = hn;
            if (fabs(dh) < p->h_rel_tol * h) { conv = 1; ++it; break; }
        }
        double rho, drho;
        int64_t c;
        density_sums(p, n, pos, m, i, h, &rho, &drho, &c);
        h_out[s] = h;
        rho_out[s] = rho;
        omega_out[s] = 1.0 + h / (3.0 * rho) * drho;
        nngb_out[s] = c;
        iters_out[s] = conv ? it : -1;
        if (!conv) failed += 1;
    }
    return failed;
}

/* rho, Omega and neighbour count at a GIVEN h (no iteration). */
void orc_density_at(const orc_params *p, int64_t n, const double *pos, const double *m,
                    int64_t ns, const int64_t *sinks, const double *h,
                    double *rho_out, double *omega_out, int64_t *nngb_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sinks ? sinks[s] : s;
        double rho, drho;
        int64_t c;
        density_sums(p, n, pos, m, i, h[s], &rho, &drho, &c);
        rho_out[s] = rho;
        omega_out[s] = 1.0 + h[s] / (3.0 * rho) * drho;
        nngb_out[s] = c;
    }
}

/*
 * Neighbours of particle i: every j != i with r_ij < h strictly.  Writes at
 * most cap indices (in increasing j) and returns the full count.
 * margin_out = min over all j != i of |r_ij - h| / h (how close the nearest
 * particle sits to the support boundary).
 */
int64_t orc_neighbours(const orc_params *p, int64_t n, const double *pos, int64_t i, double h,
                       int64_t cap, int64_t *out, double *margin_out)
{
    int64_t c = 0;
    double mg = INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        separation(p, pos + 3 * i, pos + 3 * j, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double g = fabs(r - h) / h;
        if (g < mg) mg = g;
        if (r < h) {
            if (c < cap) out[c] = j;
            ++c;
        }
    }
    *margin_out = mg;
    return c;
}

/*
 * Time derivatives for the listed sinks (Sec. 2.3.5, Sec. 2.3.6).
 * Inputs are the predicted velocity vel and internal energy u of ALL
 * particles together with h, rho, Omega from the density pass.
 *   P = (gamma-1) rho u,  c = sqrt(gamma P / rho)
 *   a_i  = - sum_j m_j [ P_i/(Om_i rho_i^2) dW_ij(h_i)/dr_i + P_j/(Om_j rho_j^2) dW_ij(h_j)/dr_i ]
 *          - sum_j m_j Pi_ij dWbar_ij/dr_i
 *   du_i/dt|H  = P_i/(Om_i rho_i^2) sum_j m_j v_ij . dW_ij(h_i)/dr_i
 *   du_i/dt|Pi = 1/2 sum_j m_j Pi_ij v_ij . dWbar_ij/dr_i
 *   Pi_ij = (-alpha cbar mu + beta mu^2)/rhobar  if v_ij . r_ij < 0, else 0
 *   mu_ij = hbar (v_ij . r_ij) / (r_ij^2 + eps hbar^2)
 *   Wbar = (W(h_i) + W(h_j))/2, bars are arithmetic means
 *   div v_i = -1/(Om_i rho_i) sum_j m_j v_ij . dW_ij(h_i)/dr_i
 *   dt_i = min( eta_a sqrt(h_i/|a_i|),
 *               eta_C min_j h_i / ((1+0.6 alpha) c_i + 0.6 beta |min(0, mu_ij)|) )
 * The sum over j covers every j != i with r_ij < max(h_i, h_j) (outside it
 * all kernel terms vanish); the CFL minimum runs over the same j and falls
 * back to the mu = 0 value when there are none.
 */
void orc_forces(const orc_params *p, int64_t n, const double *pos, const double *vel,
                const double *m, const double *h, const double *rho, const double *omega,
                const double *u, int64_t ns, const int64_t *sinks,
                double *acc_out, double *dudt_h_out, double *dudt_av_out, double *divv_out,
                double *dt_out, double *vdw_abs_out)
{
    const double g = p->gamma;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sinks ? sinks[s] : s;
        double Pi_ = (g - 1.0) * rho[i] * u[i];
        double ci = sqrt(g * Pi_ / rho[i]);
        double Ai = Pi_ / (omega[i] * rho[i] * rho[i]);
        double a[3] = {0.0, 0.0, 0.0};
        double sum_vdw = 0.0, du_av = 0.0;
        double abs_vdw = 0.0;  /* sum of |terms| of sum_vdw: its conditioning */
        double cfl = h[i] / ((1.0 + 0.6 * p->alpha) * ci);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            separation(p, pos + 3 * i, pos + 3 * j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (!(r < h[i] || r < h[j])) continue;
            double Pj = (g - 1.0) * rho[j] * u[j];
            double cj = sqrt(g * Pj / rho[j]);
            double Aj = Pj / (omega[j] * rho[j] * rho[j]);
            /* gradients of W_ij(h_i) and W_ij(h_j) with respect to x_i */
            double gi[3], gj[3];
            double fi = dWdr_of(p->kernel, r, h[i]) / r;
            double fj = dWdr_of(p->kernel, r, h[j]) / r;
            for (int a_ = 0; a_ < 3; ++a_) { gi[a_] = d[a_] * fi; gj[a_] = d[a_] * fj; }
            double vij[3] = {vel[3 * i] - vel[3 * j], vel[3 * i + 1] - vel[3 * j + 1],
                             vel[3 * i + 2] - vel[3 * j + 2]};
            /* hydro (pressure) part */
            for (int a_ = 0; a_ < 3; ++a_) a[a_] -= m[j] * (Ai * gi[a_] + Aj * gj[a_]);
            sum_vdw += m[j] * (vij[0] * gi[0] + vij[1] * gi[1] + vij[2] * gi[2]);
            abs_vdw += fabs(m[j] * (vij[0] * gi[0] + vij[1] * gi[1] + vij[2] * gi[2]));
            /* artificial viscosity */
            double vr = vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2];
            double hb = 0.5 * (h[i] + h[j]);
            double cb = 0.5 * (ci + cj);
            double rb = 0.5 * (rho[i] + rho[j]);
            double mu = hb * vr / (r * r + p->eps_av * hb * hb);
            if (vr < 0.0) {
                double PI = (-p->alpha * cb * mu + p->beta * mu * mu) / rb;
                double gb[3];
                for (int a_ = 0; a_ < 3; ++a_) gb[a_] = 0.5 * (gi[a_] + gj[a_]);
                for (int a_ = 0; a_ < 3; ++a_) a[a_] -= m[j] * PI * gb[a_];
                du_av += 0.5 * m[j] * PI * (vij[0] * gb[0] + vij[1] * gb[1] + vij[2] * gb[2]);
            }
            double mneg = mu < 0.0 ? -mu : 0.0;
            double c_ = h[i] / ((1.0 + 0.6 * p->alpha) * ci + 0.6 * p->beta * mneg);
            if (c_ < cfl) cfl = c_;
        }
        acc_out[3 * s] = a[0];
        acc_out[3 * s + 1] = a[1];
        acc_out[3 * s + 2] = a[2];
        dudt_h_out[s] = Ai * sum_vdw;
        dudt_av_out[s] = du_av;
        divv_out[s] = -sum_vdw / (omega[i] * rho[i]);
        if (vdw_abs_out) vdw_abs_out[s] = abs_vdw;
        double amag = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double dta = amag > 0.0 ? p->eta_acc * sqrt(h[i] / amag) : INFINITY;
        double dtc = p->eta_courant * cfl;
        dt_out[s] = dta < dtc ? dta : dtc;
    }
}

/*
 * Kernel imbalance of the listed sinks (Sec. 2.3.4, Eq. Kernel_imbalance):
 *   I_i = alpha |sum_j kappa_ij (r_j - r_i) m_j W_ij(h_i)| / (h_i sum_j m_j W_ij(h_i))
 * kappa_ij = +1 for particles of the same material, -1 otherwise; the sums
 * run over every j (the i = j term adds m_i W(0,h_i) to the denominator only).
 * r_j - r_i is the minimum image of x_j - x_i.
 */
void orc_imbalance(const orc_params *p, int64_t n, const double *pos, const double *m,
                   const double *h, const int32_t *mat, double alpha, int64_t ns,
                   const int64_t *sinks, double *imb_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sinks ? sinks[s] : s;
        double v[3] = {0.0, 0.0, 0.0}, den = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double d[3];
            separation(p, pos + 3 * i, pos + 3 * j, d);  /* d = r_i - r_j */
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r >= h[i]) continue;
            double w = m[j] * W_of(p->kernel, r, h[i]);
            double kappa = mat[j] == mat[i] ? 1.0 : -1.0;
            for (int a = 0; a < 3; ++a) v[a] += kappa * (-d[a]) * w;
            den += w;
        }
        double mag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        imb_out[s] = alpha * mag / (h[i] * den);
    }
}

/*
 * Kernel averages of temperature and pressure weighted by exp(-I_j^2)
 * (Sec. 2.3.4, interface correction pass):
 *   Tbar_i = sum_j T_j e^{-I_j^2} W_ij(h_i) / sum_j e^{-I_j^2} W_ij(h_i),
 *   Pbar_i likewise with P_j; every j with r_ij < h_i, i itself included.
 */
void orc_interface_averages(const orc_params *p, int64_t n, const double *pos, const double *h,
                            const double *eI, const double *T, const double *P, int64_t ns,
                            const int64_t *sinks, double *tbar_out, double *pbar_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; ++s) {
        int64_t i = sinks ? sinks[s] : s;
        double st = 0.0, sp = 0.0, sw = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double d[3];
            separation(p, pos + 3 * i, pos + 3 * j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r >= h[i]) continue;
            double w = eI[j] * W_of(p->kernel, r, h[i]);
            st += T[j] * w;
            sp += P[j] * w;
            sw += w;
        }
        tbar_out[s] = st / sw;
        pbar_out[s] = sp / sw;
    }
}

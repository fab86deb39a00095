/*
 * Plain FP64 CPU oracle for the split-operator time step of the time-dependent
 * Schroedinger equation (Dion, Hashemloo, Rahali, "Program for quantum
 * wave-packet dynamics with time-dependent potentials", arXiv:1306.3247).
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA path. Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, and where each piece comes from:
 *   - Eq. (1)-(2): i hbar dpsi/dt = (P^2/2m + V(x,t)) psi, V the sum of the
 *     potential terms plus an optional static grid (Sec. 3.2.3: the user
 *     potential() evaluated at every grid point).
 *   - Eq. (grid): x_i = x_min + i dx. This oracle uses the half-open periodic
 *     reading dx = L/n (the FFT period is n dx under either reading).
 *   - Eq. (ft) and the momentum grid of Sec. 2.1: the kinetic factor is applied
 *     in momentum space, p = hbar k, k_j = 2 pi j'/L with j' = j for j < n/2
 *     and j' = j - n otherwise (natural FFT output order).
 *   - Eq. (splitop): the symmetric split. Two orders are provided:
 *       VKV: psi <- e^{-iV(t_{n+1})dt/2hbar} F^-1 e^{-iT dt} F e^{-iV(t_n)dt/2hbar} psi,
 *            i.e. the V integral by the trapezoid rule, T = hbar |k|^2 / 2m;
 *       KVK: the paper's order, K half-step, V full step at the midpoint
 *            t_n + dt/2, K half-step.
 *     Half-steps are never merged here: each step is applied as written.
 *   - Tab. 3 and Sec. 3.2.6: norm, <x>, <x^2>, energy <psi|H|psi>,
 *     autocorrelation |<psi(0)|psi(t)>|^2, plus <p>.
 *   - Sec. 4.2: normalised Gaussian packet
 *       psi = (2/pi)^{d/4} prod_xi sigma_xi^{-1/2} e^{i p_xi0 (xi - xi0)/hbar}
 *             e^{-(xi - xi0)^2/sigma_xi^2}.
 *   - Algorithm 1: observables at step 0 and every nprint steps.
 *
 * The FFT is its own recursive radix-2 decimation-in-time transform with
 * twiddles cos/sin(2 pi k/n) in double, unnormalised, forward sign -1.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Problem and potential descriptors (the oracle's own definitions).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t ndim;        /* 1, 2 or 3; 1-D along x, 2-D in xy (Sec. 2.2) */
  int32_t order;       /* 0 = VKV, 1 = KVK (eq. splitop) */
  int64_t n[3];        /* grid points per axis (unused axes: 1) */
  double xmin[3];      /* first grid point per axis */
  double L[3];         /* period per axis; dx = L/n */
  double mass, hbar, dt, t0;
  const double *vgrid; /* optional static potential on the grid, row-major, or NULL:
                          the user potential() of Sec. 3.2.3 evaluated once */
} orc_problem;

/* One potential term: V_term(x,t) = f(t) * shape(x,t).
 * shape: 0 const (1)
 *        1 quad    0.5 * sum_d a_d (x_d - c_d(t))^2
 *        2 linear  sum_d a_d (x_d - c_d(t))
 *        3 gauss   exp(-sum_{d: a_d>0} (x_d - c_d(t))^2 / a_d^2)
 *        4 morse   a_0 * (1 - exp(-a_1 (x_axis - c_axis(t))))^2, axis = (int)a_2
 * with centre c_d(t) = c0_d + v_d t.
 * f(t) = A0 + A * env(t) * sin(omega t + phi),
 * env: 0 none (1); 1 gauss exp(-(t - t0)^2/tau^2);
 *      2 sin2: sin^2(pi t/tau) for t0 <= t <= t0 + tau, 0 otherwise (Sec. 4.1). */
typedef struct {
  int32_t shape, env;
  double a[3], c0[3], v[3];
  double A0, A, omega, phi, t0, tau;
} orc_term;

/* ---------------------------------------------------------------------------
 * FFT: recursive radix-2 decimation in time.
 * X_k = sum_j x_j exp(sign * 2 pi i j k / n), n a power of two.
 * work must hold at least 2n entries.
 * ------------------------------------------------------------------------- */
static void fft_rec(cplx *a, int64_t n, int sign, cplx *work) {
  if (n == 1) return;
  int64_t h = n / 2;
  cplx *even = work, *odd = work + h;
  for (int64_t i = 0; i < h; i++) {
    even[i] = a[2 * i];
    odd[i] = a[2 * i + 1];
  }
  fft_rec(even, h, sign, work + n);
  fft_rec(odd, h, sign, work + n);
  for (int64_t k = 0; k < h; k++) {
    double ang = 2.0 * ORC_PI * (double)k / (double)n;
    double wr = cos(ang), wi = sign * sin(ang);
    double orr = creal(odd[k]), oi = cimag(odd[k]);
    double tr = wr * orr - wi * oi, ti = wr * oi + wi * orr;
    double er = creal(even[k]), ei = cimag(even[k]);
    a[k] = CMPLX(er + tr, ei + ti);
    a[k + h] = CMPLX(er - tr, ei - ti);
  }
}

void orc_fft1d(cplx *a, int64_t n, int sign) {
  cplx *work = (cplx *)malloc(sizeof(cplx) * 2 * (size_t)n + 16);
  fft_rec(a, n, sign, work);
  free(work);
}

/* Multi-dimensional FFT on a row-major [n0][n1][n2] array (last axis fastest):
 * the 1-D transform applied along every axis in turn. */
void orc_fftnd(cplx *psi, int32_t ndim, const int64_t *n, int sign) {
  int64_t ext[3] = {1, 1, 1};
  for (int d = 0; d < ndim; d++) ext[d] = n[d];
  for (int d = 0; d < ndim; d++) {
    int64_t len = ext[d];
    if (len == 1) continue;
    int64_t inner = 1;
    for (int e = d + 1; e < 3; e++) inner *= ext[e];
    int64_t outer = 1;
    for (int e = 0; e < d; e++) outer *= ext[e];
    int64_t nlines = outer * inner;
#pragma omp parallel
    {
      cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)len);
      cplx *work = (cplx *)malloc(sizeof(cplx) * 2 * (size_t)len + 16);
#pragma omp for schedule(static)
      for (int64_t l = 0; l < nlines; l++) {
        int64_t o = l / inner, c = l % inner;
        cplx *base = psi + o * len * inner + c;
        for (int64_t i = 0; i < len; i++) line[i] = base[i * inner];
        fft_rec(line, len, sign, work);
        for (int64_t i = 0; i < len; i++) base[i * inner] = line[i];
      }
      free(line);
      free(work);
    }
  }
}

/* ---------------------------------------------------------------------------
 * Grid helpers.
 * ------------------------------------------------------------------------- */
static int64_t ext_of(const orc_problem *p, int d) { return d < p->ndim ? p->n[d] : 1; }

static int64_t total_points(const orc_problem *p) {
  return ext_of(p, 0) * ext_of(p, 1) * ext_of(p, 2);
}

static double coord(const orc_problem *p, int d, int64_t i) {
  return p->xmin[d] + (double)i * (p->L[d] / (double)p->n[d]);
}

/* Wave number of FFT output index j on axis d (natural FFT order). */
static double wavenumber(const orc_problem *p, int d, int64_t j) {
  int64_t n = p->n[d];
  int64_t js = (j < n / 2) ? j : j - n;
  return 2.0 * ORC_PI * (double)js / p->L[d];
}

static double cell_volume(const orc_problem *p) {
  double v = 1.0;
  for (int d = 0; d < p->ndim; d++) v *= p->L[d] / (double)p->n[d];
  return v;
}

/* ---------------------------------------------------------------------------
 * Potential V(x,t), the user potential() of Sec. 3.2.3 written as a sum of terms.
 * ------------------------------------------------------------------------- */
static double term_coef(const orc_term *tm, double t) {
  double env = 1.0;
  if (tm->env == 1) {
    double u = (t - tm->t0) / tm->tau;
    env = exp(-u * u);
  } else if (tm->env == 2) {
    if (t >= tm->t0 && t <= tm->t0 + tm->tau) {
      double s = sin(ORC_PI * t / tm->tau);
      env = s * s;
    } else {
      env = 0.0;
    }
  }
  return tm->A0 + tm->A * env * sin(tm->omega * t + tm->phi);
}

static double term_shape(const orc_term *tm, int ndim, const double *x, double t) {
  double r = 0.0;
  switch (tm->shape) {
    case 0:
      return 1.0;
    case 1:
      for (int d = 0; d < ndim; d++) {
        double u = x[d] - (tm->c0[d] + tm->v[d] * t);
        r += 0.5 * tm->a[d] * u * u;
      }
      return r;
    case 2:
      for (int d = 0; d < ndim; d++) r += tm->a[d] * (x[d] - (tm->c0[d] + tm->v[d] * t));
      return r;
    case 3:
      for (int d = 0; d < ndim; d++) {
        if (tm->a[d] > 0.0) {
          double u = (x[d] - (tm->c0[d] + tm->v[d] * t)) / tm->a[d];
          r += u * u;
        }
      }
      return exp(-r);
    case 4: {
      int ax = (int)tm->a[2];
      double u = x[ax] - (tm->c0[ax] + tm->v[ax] * t);
      double e = 1.0 - exp(-tm->a[1] * u);
      return tm->a[0] * e * e;
    }
  }
  return 0.0;
}

double orc_potential_at(const orc_problem *p, int32_t nterms, const orc_term *terms,
                        const double *x, double t) {
  double v = 0.0;
  for (int k = 0; k < nterms; k++) v += term_coef(&terms[k], t) * term_shape(&terms[k], p->ndim, x, t);
  return v;
}

/* V on every grid point at time t, row-major. */
void orc_potential_grid(const orc_problem *p, int32_t nterms, const orc_term *terms, double t,
                        double *out) {
  int64_t n0 = ext_of(p, 0), n1 = ext_of(p, 1), n2 = ext_of(p, 2);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        double x[3] = {coord(p, 0, i), p->ndim > 1 ? coord(p, 1, j) : 0.0,
                       p->ndim > 2 ? coord(p, 2, k) : 0.0};
        int64_t idx = (i * n1 + j) * n2 + k;
        out[idx] = orc_potential_at(p, nterms, terms, x, t) + (p->vgrid ? p->vgrid[idx] : 0.0);
      }
}

/* psi <- exp(-i V(x,t) tau / hbar) psi */
static void apply_potential_phase(const orc_problem *p, int32_t nterms, const orc_term *terms,
                                  cplx *psi, double t, double tau) {
  int64_t n0 = ext_of(p, 0), n1 = ext_of(p, 1), n2 = ext_of(p, 2);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        double x[3] = {coord(p, 0, i), p->ndim > 1 ? coord(p, 1, j) : 0.0,
                       p->ndim > 2 ? coord(p, 2, k) : 0.0};
        int64_t idx = (i * n1 + j) * n2 + k;
        double v = orc_potential_at(p, nterms, terms, x, t) + (p->vgrid ? p->vgrid[idx] : 0.0);
        double th = -v * tau / p->hbar;
        psi[idx] = psi[idx] * CMPLX(cos(th), sin(th));
      }
}

/* psi_hat <- exp(-i hbar |k|^2 tau / 2m) psi_hat / N : the kinetic factor of
 * eq. (ft) with the 1/N of the unnormalised inverse FFT folded in. */
static void apply_kinetic_phase(const orc_problem *p, cplx *psih, double tau) {
  int64_t n0 = ext_of(p, 0), n1 = ext_of(p, 1), n2 = ext_of(p, 2);
  double inv_n = 1.0 / (double)total_points(p);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        double k2 = 0.0, kk;
        kk = wavenumber(p, 0, i);
        k2 += kk * kk;
        if (p->ndim > 1) {
          kk = wavenumber(p, 1, j);
          k2 += kk * kk;
        }
        if (p->ndim > 2) {
          kk = wavenumber(p, 2, k);
          k2 += kk * kk;
        }
        double th = -p->hbar * k2 * tau / (2.0 * p->mass);
        int64_t idx = (i * n1 + j) * n2 + k;
        psih[idx] = psih[idx] * CMPLX(cos(th), sin(th)) * inv_n;
      }
}

/* One kinetic propagation exp(-i K tau/hbar) = F^-1 e^{-i T tau} F (eq. ft). */
static void kinetic_step(const orc_problem *p, cplx *psi, double tau) {
  orc_fftnd(psi, p->ndim, p->n, -1);
  apply_kinetic_phase(p, psi, tau);
  orc_fftnd(psi, p->ndim, p->n, +1);
}

/* Time of step index s: t_s = t0 + s dt, a product, never a running sum. */
static double time_of(const orc_problem *p, int64_t s) { return p->t0 + (double)s * p->dt; }

/* One Strang step from step index s to s+1. */
void orc_step(const orc_problem *p, int32_t nterms, const orc_term *terms, cplx *psi, int64_t s) {
  double dt = p->dt;
  if (p->order == 0) {
    apply_potential_phase(p, nterms, terms, psi, time_of(p, s), 0.5 * dt);
    kinetic_step(p, psi, dt);
    apply_potential_phase(p, nterms, terms, psi, time_of(p, s + 1), 0.5 * dt);
  } else {
    kinetic_step(p, psi, 0.5 * dt);
    apply_potential_phase(p, nterms, terms, psi, time_of(p, s) + 0.5 * dt, dt);
    kinetic_step(p, psi, 0.5 * dt);
  }
}

/* ---------------------------------------------------------------------------
 * Observables (Tab. 3, Sec. 3.2.6). Record layout, 16 doubles:
 *  0 t, 1 norm, 2-4 <x_d>, 5-7 <p_d>, 8-10 <x_d^2>, 11 energy, 12 kinetic,
 *  13 potential, 14 autocorrelation, 15 step index.
 * Expectation values are the plain integrals <psi|A|psi>, not divided by the
 * norm, as expectation1D and the energy flag define them.
 * ------------------------------------------------------------------------- */
void orc_observe(const orc_problem *p, int32_t nterms, const orc_term *terms, const cplx *psi,
                 const cplx *psi0, int64_t s, double *rec) {
  int64_t n0 = ext_of(p, 0), n1 = ext_of(p, 1), n2 = ext_of(p, 2);
  int64_t N = n0 * n1 * n2;
  double dv = cell_volume(p);
  double t = time_of(p, s);
  double s0 = 0, sx[3] = {0, 0, 0}, sxx[3] = {0, 0, 0}, sv = 0;
  double acr = 0, aci = 0;
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        int64_t idx = (i * n1 + j) * n2 + k;
        double x[3] = {coord(p, 0, i), p->ndim > 1 ? coord(p, 1, j) : 0.0,
                       p->ndim > 2 ? coord(p, 2, k) : 0.0};
        double rho = creal(psi[idx]) * creal(psi[idx]) + cimag(psi[idx]) * cimag(psi[idx]);
        s0 += rho;
        for (int d = 0; d < p->ndim; d++) {
          sx[d] += x[d] * rho;
          sxx[d] += x[d] * x[d] * rho;
        }
        sv += (orc_potential_at(p, nterms, terms, x, t) + (p->vgrid ? p->vgrid[idx] : 0.0)) * rho;
        if (psi0) {
          cplx c = conj(psi0[idx]) * psi[idx];
          acr += creal(c);
          aci += cimag(c);
        }
      }
  cplx *ph = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  memcpy(ph, psi, sizeof(cplx) * (size_t)N);
  orc_fftnd(ph, p->ndim, p->n, -1);
  double sp[3] = {0, 0, 0}, sk2 = 0;
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        int64_t idx = (i * n1 + j) * n2 + k;
        double rho = creal(ph[idx]) * creal(ph[idx]) + cimag(ph[idx]) * cimag(ph[idx]);
        int64_t ij[3] = {i, j, k};
        for (int d = 0; d < p->ndim; d++) {
          double kk = wavenumber(p, d, ij[d]);
          sp[d] += kk * rho;
          sk2 += kk * kk * rho;
        }
      }
  free(ph);
  double dvk = dv / (double)N; /* Parseval for the unnormalised transform */
  memset(rec, 0, 16 * sizeof(double));
  rec[0] = t;
  rec[1] = sqrt(s0 * dv);
  for (int d = 0; d < p->ndim; d++) {
    rec[2 + d] = sx[d] * dv;
    rec[5 + d] = p->hbar * sp[d] * dvk;
    rec[8 + d] = sxx[d] * dv;
  }
  rec[12] = p->hbar * p->hbar / (2.0 * p->mass) * sk2 * dvk;
  rec[13] = sv * dv;
  rec[11] = rec[12] + rec[13];
  rec[14] = psi0 ? (acr * acr + aci * aci) * dv * dv : 0.0;
  rec[15] = (double)s;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 run loop: observables at step s0 and at every multiple of nprint
 * after it; all nt steps run even when nprint does not divide nt.
 * obs must hold 1 + nt/nprint records. Returns the number written, or -1 on
 * nprint > nt (Sec. 3.4: the program refuses that input).
 * ------------------------------------------------------------------------- */
int64_t orc_run(const orc_problem *p, int32_t nterms, const orc_term *terms, cplx *psi,
                int64_t s0, int64_t nt, int64_t nprint, double *obs) {
  if (nprint <= 0 || nprint > nt) return -1;
  int64_t N = total_points(p);
  cplx *psi0 = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  memcpy(psi0, psi, sizeof(cplx) * (size_t)N);
  int64_t nobs = 0;
  if (obs) orc_observe(p, nterms, terms, psi, psi0, s0, obs + 16 * nobs++);
  for (int64_t s = 0; s < nt; s++) {
    orc_step(p, nterms, terms, psi, s0 + s);
    if (obs && (s + 1) % nprint == 0) orc_observe(p, nterms, terms, psi, psi0, s0 + s + 1, obs + 16 * nobs++);
  }
  free(psi0);
  return nobs;
}

/* Plain propagation without observables. */
void orc_propagate(const orc_problem *p, int32_t nterms, const orc_term *terms, cplx *psi,
                   int64_t s0, int64_t nt) {
  for (int64_t s = 0; s < nt; s++) orc_step(p, nterms, terms, psi, s0 + s);
}

/* Normalised Gaussian packet of Sec. 4.2 on the grid. */
void orc_gaussian(const orc_problem *p, const double *x0, const double *p0, const double *sigma,
                  cplx *psi) {
  int64_t n0 = ext_of(p, 0), n1 = ext_of(p, 1), n2 = ext_of(p, 2);
  double pref = pow(2.0 / ORC_PI, 0.25 * p->ndim);
  for (int d = 0; d < p->ndim; d++) pref /= sqrt(sigma[d]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n0; i++)
    for (int64_t j = 0; j < n1; j++)
      for (int64_t k = 0; k < n2; k++) {
        int64_t ij[3] = {i, j, k};
        cplx v = pref;
        for (int d = 0; d < p->ndim; d++) {
          double u = coord(p, d, ij[d]) - x0[d];
          double ph = p0[d] * u / p->hbar;
          v *= CMPLX(cos(ph), sin(ph)) * exp(-u * u / (sigma[d] * sigma[d]));
        }
        psi[(i * n1 + j) * n2 + k] = v;
      }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

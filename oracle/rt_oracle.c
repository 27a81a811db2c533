/*
 * FP64 CPU oracle of the frequency-dependent first-order stellar irradiation
 * ray tracer of Kuiper, Klahr, Dullemond, Kley & Henning (2010):
 *   Sect. 2.2, Eqs. 17-19  (attenuated stellar flux along radial rays),
 *   Sect. 2.3, Eq. 20      (per-bin stellar boundary flux, kappa(nu) per bin),
 *   Sect. 3.3.4, Eqs. 27-36 (cell-integrated absorption / radiative force).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this code. The CUDA library never links, includes or
 * calls it, and it shares no code, header, table or constant with the library.
 *
 * It is written to be checked against the paper by eye, not to be fast: for every
 * ray, every frequency bin and every cell it evaluates the definition with libm
 * exp/expm1 in double precision, in the order bins ascending, cells outward.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - Eq. 20 is read as F_i = pi * int B_nu dnu over the bin (B_nu the specific
 *    intensity), so that sum_i F_i = sigma T^4, consistent with Eq. 18 and
 *    sigma = a c / 4.
 *  - Bin edges are arithmetic midpoints of neighbouring mid-frequencies; the
 *    lowest bin starts at nu = 0 and the highest ends at nu = infinity.
 *  - tau = 0 at the inner grid radius (Sect. 2.2, optical depth between the star
 *    and the inner boundary neglected); geometric dilution (R_s/r)^2 of a point
 *    source evaluated at the interface radius (Eq. 17).
 *  - kappa_nu is zero in a cell whose dust temperature exceeds t_sub (evaporated
 *    dust, Sect. 2); a cell at exactly t_sub keeps its dust.
 *  - Temperature-dependent tables (rto_irradiate_tdep, an extension the paper's
 *    "tabulated dust opacities" allow): kappa_i linear in T between grid points.
 *  - Absorbed power of cell k in bin i (Eqs. 28-32 carried to spherical shells,
 *    Eq. 36): P = F_i R_s^2 dOmega exp(-tau_in) (-expm1(-dtau)), dtau = kappa rho dr.
 *  - a_rad = -div(F_s)/(rho c) (Sect. 5) written without the division by rho:
 *    sum_i F_i R_s^2 dOmega exp(-tau_in) kappa_i dr phi(dtau) / (V c),
 *    phi(x) = -expm1(-x)/x, phi(0) = 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact SI values, expressed in cgs */
static const double RTO_C = 2.99792458e10;     /* cm s^-1 */
static const double RTO_H = 6.62607015e-27;    /* erg s */
static const double RTO_K = 1.380649e-16;      /* erg K^-1 */
static const double RTO_PI = 3.14159265358979323846;

double rto_sigma_sb(void)
{
    /* Stefan-Boltzmann constant sigma = 2 pi^5 k^4 / (15 h^3 c^2) */
    return 2.0 * pow(RTO_PI, 5) * pow(RTO_K, 4) / (15.0 * pow(RTO_H, 3) * RTO_C * RTO_C);
}

/* ---------------------------------------------------------------------------
 * Planck integrals in x = h nu / (k T)
 *   H(x) = int_0^x t^3/(e^t - 1) dt,   G(x) = int_x^inf t^3/(e^t - 1) dt,
 *   H(inf) = G(0) = pi^4 / 15.
 * ------------------------------------------------------------------------- */

/* H(x) for 0 <= x <= 1 from t/(e^t-1) = sum_n B_n t^n / n! (radius 2 pi):
 * t^3/(e^t-1) = sum_n B_n t^(n+2) / n!, integrated term by term. */
double rto_planck_H_small(double x)
{
    /* Bernoulli numbers B_0..B_22 (B_1 = -1/2, odd ones above 1 vanish) */
    static const double bern_even[12] = {
        1.0, 1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0,
        -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0, 43867.0 / 798.0,
        -174611.0 / 330.0, 854513.0 / 138.0};
    double sum = x * x * x / 3.0 - x * x * x * x / 8.0; /* n = 0 and n = 1 */
    double fact = 1.0;                                   /* n! */
    for (int n = 2; n <= 22; n += 2) {
        fact *= (double)(n - 1) * (double)n;
        sum += bern_even[n / 2] * pow(x, n + 3) / (fact * (double)(n + 3));
    }
    return sum;
}

/* G(x) for x >= 1 from 1/(e^t-1) = sum_{m>=1} e^{-m t}, each term integrated:
 * int_x^inf t^3 e^{-m t} dt = e^{-m x} (x^3/m + 3 x^2/m^2 + 6 x/m^3 + 6/m^4). */
double rto_planck_G_large(double x)
{
    double sum = 0.0;
    for (int m = 1; m <= 200; ++m) {
        double dm = (double)m;
        double term = exp(-dm * x) *
                      (x * x * x / dm + 3.0 * x * x / (dm * dm) + 6.0 * x / (dm * dm * dm) +
                       6.0 / (dm * dm * dm * dm));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* int_a^b t^3/(e^t-1) dt for 0 <= a < b <= inf, evaluated without subtracting
 * two nearly equal totals: H differences below x = 1, G differences above. */
double rto_planck_band(double a, double b)
{
    const double total = pow(RTO_PI, 4) / 15.0;
    if (isinf(b)) {
        if (a >= 1.0) return rto_planck_G_large(a);
        return total - rto_planck_H_small(a);
    }
    if (b <= 1.0) return rto_planck_H_small(b) - rto_planck_H_small(a);
    if (a >= 1.0) return rto_planck_G_large(a) - rto_planck_G_large(b);
    return (rto_planck_H_small(1.0) - rto_planck_H_small(a)) +
           (rto_planck_G_large(1.0) - rto_planck_G_large(b));
}

/* Eq. 20 (read as F_i = pi int B_nu dnu over the bin):
 * F_i = (2 pi k^4 T^4 / (h^3 c^2)) int_{x_lo}^{x_hi} t^3/(e^t-1) dt,
 * bin edges at arithmetic midpoints of mid-frequencies, outer edges 0 and inf.
 * Returns 0, or -1 on a bad argument. */
int rto_planck_bins(double t_star, int n_nu, const double *nu_mid, double *f_bin)
{
    if (!(t_star > 0.0) || n_nu < 1) return -1;
    for (int i = 0; i < n_nu; ++i)
        if (!(nu_mid[i] > 0.0) || (i > 0 && !(nu_mid[i] > nu_mid[i - 1]))) return -1;
    const double kt_over_h = RTO_K * t_star / RTO_H;
    const double pref = 2.0 * RTO_PI * pow(RTO_K * t_star, 4) / (pow(RTO_H, 3) * RTO_C * RTO_C);
    for (int i = 0; i < n_nu; ++i) {
        double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);
        double hi = (i == n_nu - 1) ? INFINITY : 0.5 * (nu_mid[i] + nu_mid[i + 1]);
        double xlo = lo / kt_over_h;
        double xhi = isinf(hi) ? INFINITY : hi / kt_over_h;
        f_bin[i] = pref * rto_planck_band(xlo, xhi);
    }
    return 0;
}

/* Planck mean opacity of a bin table at temperature t (kappa_P(T) of Eq. 16):
 * sum_i kappa_i B_i(t) / sum_i B_i(t), B_i the Planck integral over bin i with the
 * bin edges of Eq. 20. Returns a negative value on a bad argument. */
double rto_planck_mean(double t, int n_nu, const double *nu_mid, const double *kappa)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)(n_nu > 0 ? n_nu : 1));
    if (!f) return -1.0;
    if (rto_planck_bins(t, n_nu, nu_mid, f) != 0) {
        free(f);
        return -1.0;
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n_nu; ++i) {
        num += kappa[i] * f[i];
        den += f[i];
    }
    free(f);
    return den > 0.0 ? num / den : 0.0;
}

/* Rosseland mean opacity of a bin table at temperature t (the kappa_R of the FLD
 * diffusion constant, Eq. 11): 1/kappa_R = sum_i W_i / kappa_i / sum_i W_i with
 * W_i = int over bin i of dB_nu/dT dnu. In x = h nu / (k T) the weight is
 * int t^4 e^t / (e^t - 1)^2 dt, and by parts (d/dt of 1/(e^t - 1) is
 * -e^t/(e^t - 1)^2) over [a, b]:
 *     a^4/(e^a - 1) - b^4/(e^b - 1) + 4 int_a^b t^3/(e^t - 1) dt.
 * A bin with kappa = 0 and weight > 0 makes the mean 0. Returns < 0 on a bad
 * argument. */
double rto_rosseland_mean(double t, int n_nu, const double *nu_mid, const double *kappa)
{
    if (!(t > 0.0) || n_nu < 1) return -1.0;
    const double kt_over_h = RTO_K * t / RTO_H;
    double num = 0.0, den = 0.0;
    int opaque_gap = 0;
    for (int i = 0; i < n_nu; ++i) {
        double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);
        double hi = (i == n_nu - 1) ? INFINITY : 0.5 * (nu_mid[i] + nu_mid[i + 1]);
        const double a = lo / kt_over_h, b = isinf(hi) ? INFINITY : hi / kt_over_h;
        const double ea = (a > 0.0) ? pow(a, 4) / expm1(a) : 0.0;
        const double eb = (isinf(b) || b > 700.0) ? 0.0 : pow(b, 4) / expm1(b);
        const double w = ea - eb + 4.0 * rto_planck_band(a, b);
        den += w;
        if (kappa[i] > 0.0) num += w / kappa[i];
        else if (w > 0.0) opaque_gap = 1;
    }
    if (opaque_gap || !(num > 0.0)) return 0.0;
    return den / num;
}

/* Eq. 16 with frequency-dependent fluxes, per cell: the dust temperature T with
 *     a T^4 = E_R + a_rad / kappa_P(T),   a = 4 sigma / c,
 * (sum_i kappa_i F_i over the cell is q_abs / rho = c a_rad). kappa_P is evaluated
 * at T clamped to [t_lo, t_hi]. Bisection on ln T over [ln 1e-3, ln 1e9] until the
 * bracket is 1e-14 wide in ln T; T = 0 where a_rad = E_R = 0. e_rad may be NULL
 * (E_R = 0). Returns 0, or -1 on a bad argument. */
int rto_dust_temperature(long long n, const double *a_rad, const double *e_rad, double t_lo, double t_hi,
                         int n_nu, const double *nu_mid, const double *kappa, double *t_out, int nthreads)
{
    if (n < 0 || !a_rad || !t_out || n_nu < 1 || !(t_lo > 0.0) || !(t_hi > t_lo)) return -1;
    const double a_rad_const = 4.0 * rto_sigma_sb() / RTO_C;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long long c = 0; c < n; ++c) {
        const double ar = a_rad[c] > 0.0 ? a_rad[c] : 0.0;
        const double er = (e_rad && e_rad[c] > 0.0) ? e_rad[c] : 0.0;
        if (ar == 0.0 && er == 0.0) {
            t_out[c] = 0.0;
            continue;
        }
        double ylo = log(1e-3), yhi = log(1e9);
        while (yhi - ylo > 1e-14) {
            const double y = 0.5 * (ylo + yhi);
            double tt = exp(y);
            const double tk = tt < t_lo ? t_lo : (tt > t_hi ? t_hi : tt);
            const double kp = rto_planck_mean(tk, n_nu, nu_mid, kappa);
            const double f = a_rad_const * tt * tt * tt * tt - er - ar / kp;
            if (f > 0.0) yhi = y;
            else ylo = y;
        }
        t_out[c] = exp(0.5 * (ylo + yhi));
    }
    (void)nthreads;
    return 0;
}

/* Neumaier-compensated running sum */
typedef struct { double s, c; } rto_sum;
static void rto_add(rto_sum *acc, double x)
{
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
    else acc->c += (x - t) + acc->s;
    acc->s = t;
}
static double rto_total(const rto_sum *acc) { return acc->s + acc->c; }

/* phi(x) = (1 - e^{-x}) / x with phi(0) = 1 */
static double rto_phi(double x) { return x > 0.0 ? -expm1(-x) / x : 1.0; }

/*
 * The ray tracer, one ray (theta_j, phi_l) at a time.
 *
 * Fields are [nphi][ntheta][nr] with r fastest. For every ray j and bin i:
 *   dtau_{i,k}  = kappa_i [T_k <= t_sub] rho_k (r_{k+1/2} - r_{k-1/2})
 *   tau_in(k)   = sum_{k' < k} dtau_{i,k'},  tau_in(0) = 0           (Eq. 19)
 *   P_{i,k}     = F_i R_s^2 dOmega_j e^{-tau_in} (-expm1(-dtau))       (Eqs. 17, 28-32, 36)
 *   q_abs(k)    = sum_i P_{i,k} / V_k,  V_k = dOmega_j (r+^3 - r-^3)/3
 *   a_rad(k)    = sum_i F_i R_s^2 dOmega_j e^{-tau_in} kappa_i [T<=t_sub] dr phi(dtau) / (V_k c)
 *   P_esc,j     = sum_i F_i R_s^2 dOmega_j e^{-tau_total}
 * with dOmega_j = (cos theta_- - cos theta_+) (phi_+ - phi_-).
 *
 * Optional outputs (NULL to skip): p_abs [cells] absorbed power (erg/s),
 * flux_if [rays][nr+1] stellar flux at every radial interface (Eq. 17 summed over
 * bins), p_esc [rays] escaping power.
 * energy[4] = {E_abs, E_esc, L_grid, (E_abs+E_esc)/L_grid - 1}, where L_grid is
 * R_s^2 sigma T*^4 sum_j dOmega_j (= 4 pi R_s^2 sigma T*^4 on the full sphere);
 * sums are Neumaier-compensated, ray partials added in ray order.
 * Returns 0, or -1 on a bad argument.
 */
/* kappa of bin row `row` (n_t values on t_grid) at dust temperature t: linear in T
 * between the two bracketing grid points, the end values beyond the grid. With
 * n_t == 1 the opacity does not depend on T. */
static double rto_kappa_at(const double *row, int n_t, const double *t_grid, double t)
{
    if (n_t == 1 || t <= t_grid[0]) return row[0];
    if (t >= t_grid[n_t - 1]) return row[n_t - 1];
    int j = 0;
    while (!(t < t_grid[j + 1])) ++j;
    const double w = (t - t_grid[j]) / (t_grid[j + 1] - t_grid[j]);
    return row[j] + (row[j + 1] - row[j]) * w;
}

static int rto_irradiate_impl(int nr, int ntheta, int nphi,
                              const double *r_if, const double *theta_if, const double *phi_if,
                              double t_star, double r_star,
                              int n_nu, const double *nu_mid, int n_t, const double *t_grid,
                              const double *kappa, double t_sub,
                              const double *rho, const double *tdust,
                              double *q_abs, double *a_rad,
                              double *p_abs, double *flux_if, double *p_esc,
                              double *energy, int nthreads)
{
    if (nr < 1 || ntheta < 1 || nphi < 1 || n_nu < 1 || n_t < 1 || !(r_star > 0.0)) return -1;
    if (!(r_if[0] > 0.0)) return -1;
    for (int k = 0; k < nr; ++k) if (!(r_if[k + 1] > r_if[k])) return -1;
    for (int i = 0; i < n_nu * n_t; ++i) if (!(kappa[i] >= 0.0)) return -1;
    for (int j = 1; j < n_t; ++j) if (!(t_grid[j] > t_grid[j - 1])) return -1;

    double *f_bin = (double *)malloc(sizeof(double) * (size_t)n_nu);
    if (!f_bin) return -1;
    if (rto_planck_bins(t_star, n_nu, nu_mid, f_bin) != 0) { free(f_bin); return -1; }

    const long nrays = (long)ntheta * nphi;
    double *ray_abs = (double *)calloc((size_t)nrays, sizeof(double));
    double *ray_esc = (double *)calloc((size_t)nrays, sizeof(double));
    double *ray_dom = (double *)calloc((size_t)nrays, sizeof(double));
    if (!ray_abs || !ray_esc || !ray_dom) {
        free(f_bin); free(ray_abs); free(ray_esc); free(ray_dom); return -1;
    }
    const double r2 = r_star * r_star;
    if (nthreads < 1) nthreads = 1;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
#endif
    for (long j = 0; j < nrays; ++j) {
        const int it = (int)(j % ntheta);
        const int ip = (int)(j / ntheta);
        const double domega = (cos(theta_if[it]) - cos(theta_if[it + 1])) *
                              (phi_if[ip + 1] - phi_if[ip]);
        const double *rho_ray = rho + (size_t)j * nr;
        const double *t_ray = tdust + (size_t)j * nr;
        double *P = (double *)calloc((size_t)nr, sizeof(double));   /* sum_i P_{i,k} */
        double *A = (double *)calloc((size_t)nr, sizeof(double));   /* force numerator */
        double *Fif = (double *)calloc((size_t)nr + 1, sizeof(double));
        rto_sum esc = {0.0, 0.0};

        for (int i = 0; i < n_nu; ++i) {
            const double lum = f_bin[i] * r2 * domega; /* F_i R_s^2 dOmega: power into the ray */
            double tau = 0.0;
            for (int k = 0; k < nr; ++k) {
                const double dr = r_if[k + 1] - r_if[k];
                const double kap = (t_ray[k] <= t_sub) ? rto_kappa_at(kappa + (size_t)i * n_t, n_t, t_grid, t_ray[k]) : 0.0;
                const double dtau = kap * rho_ray[k] * dr;
                const double att = exp(-tau);
                Fif[k] += f_bin[i] * (r2 / (r_if[k] * r_if[k])) * att;
                P[k] += lum * att * (-expm1(-dtau));
                A[k] += lum * att * kap * dr * rto_phi(dtau);
                tau += dtau;
            }
            Fif[nr] += f_bin[i] * (r2 / (r_if[nr] * r_if[nr])) * exp(-tau);
            rto_add(&esc, lum * exp(-tau));
        }

        rto_sum absd = {0.0, 0.0};
        for (int k = 0; k < nr; ++k) {
            const double vol = domega * (pow(r_if[k + 1], 3) - pow(r_if[k], 3)) / 3.0;
            const size_t c = (size_t)j * nr + k;
            q_abs[c] = P[k] / vol;
            a_rad[c] = A[k] / (vol * RTO_C);
            if (p_abs) p_abs[c] = P[k];
            rto_add(&absd, P[k]);
        }
        if (flux_if) memcpy(flux_if + (size_t)j * (nr + 1), Fif, sizeof(double) * (size_t)(nr + 1));
        ray_abs[j] = rto_total(&absd);
        ray_esc[j] = rto_total(&esc);
        ray_dom[j] = domega;
        if (p_esc) p_esc[j] = ray_esc[j];
        free(P); free(A); free(Fif);
    }

    rto_sum e_abs = {0.0, 0.0}, e_esc = {0.0, 0.0}, dom = {0.0, 0.0};
    for (long j = 0; j < nrays; ++j) {
        rto_add(&e_abs, ray_abs[j]);
        rto_add(&e_esc, ray_esc[j]);
        rto_add(&dom, ray_dom[j]);
    }
    if (energy) {
        const double l_grid = r2 * rto_sigma_sb() * pow(t_star, 4) * rto_total(&dom);
        energy[0] = rto_total(&e_abs);
        energy[1] = rto_total(&e_esc);
        energy[2] = l_grid;
        energy[3] = (energy[0] + energy[1]) / l_grid - 1.0;
    }
    free(f_bin); free(ray_abs); free(ray_esc); free(ray_dom);
    return 0;
}

int rto_irradiate(int nr, int ntheta, int nphi,
                  const double *r_if, const double *theta_if, const double *phi_if,
                  double t_star, double r_star,
                  int n_nu, const double *nu_mid, const double *kappa, double t_sub,
                  const double *rho, const double *tdust,
                  double *q_abs, double *a_rad,
                  double *p_abs, double *flux_if, double *p_esc,
                  double *energy, int nthreads)
{
    return rto_irradiate_impl(nr, ntheta, nphi, r_if, theta_if, phi_if, t_star, r_star, n_nu, nu_mid, 1, NULL,
                              kappa, t_sub, rho, tdust, q_abs, a_rad, p_abs, flux_if, p_esc, energy, nthreads);
}

/* rto_irradiate with temperature-dependent opacities: kappa_t [n_nu][n_t] on the
 * increasing temperature grid t_grid [n_t]; each cell's kappa of bin i is that row
 * at the cell's dust temperature (rto_kappa_at), zero above t_sub. */
int rto_irradiate_tdep(int nr, int ntheta, int nphi,
                       const double *r_if, const double *theta_if, const double *phi_if,
                       double t_star, double r_star,
                       int n_nu, const double *nu_mid, int n_t, const double *t_grid,
                       const double *kappa_t, double t_sub,
                       const double *rho, const double *tdust,
                       double *q_abs, double *a_rad,
                       double *p_abs, double *flux_if, double *p_esc,
                       double *energy, int nthreads)
{
    if (n_t < 2 || !t_grid) return -1;
    return rto_irradiate_impl(nr, ntheta, nphi, r_if, theta_if, phi_if, t_star, r_star, n_nu, nu_mid, n_t, t_grid,
                              kappa_t, t_sub, rho, tdust, q_abs, a_rad, p_abs, flux_if, p_esc, energy, nthreads);
}

int rto_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

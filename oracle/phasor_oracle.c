/*
 * FP64 CPU oracle for the four phasor sums of GeRaF's lensless RF rendering.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this file's library; the CUDA product
 * path never does. It shares no code, header or constant with the CUDA path.
 *
 * Every loop nest below is the plain definition written out: one cos/sin per
 * (point or voxel, antenna, frequency) term, FP64 everywhere, sums in index
 * order, no recurrence, no blocking, no compensation. OpenMP only splits the
 * outer loop that the paper's Algorithms 1 and 2 mark "parallel".
 *
 * Notation (paper section 3, Eq. fmcw; section 5.1, Eq. ref_sim; App. A.5):
 *   antenna i at a_i, point (or voxel) x_j, r_ij = |x_j - a_i|,
 *   round-trip delay tau_ij = 2 r_ij / c,
 *   stepped frequency f_n = f0 + n*df (the FMCW sample n seen as frequency f + k t_n),
 *   phase phi_ijn = 2*pi*f_n*tau_ij.
 * Complex arrays are split into separate real and imaginary planes, row-major
 * [n_ant][n_f].
 */
#include <math.h>
#include <stddef.h>

static const double C_LIGHT = 299792458.0; /* exact SI value, m/s */
static const double TWO_PI = 6.283185307179586476925286766559;

/* Monostatic directional factor (section 3 "Reflections", App. A.3): with the
 * incoming direction w_i and the return direction w_r = -w_i, the shifted
 * Lambertian factor (w_o . w_r) with w_o = w_i - 2 (n . w_i) n equals
 * 2 (n . w_i)^2 - 1; negative values give no returned power and clamp to 0.
 * A zero normal marks an isotropic scatterer (factor 1). */
static double directional_factor(double gx, double gy, double gz,
                                 double dx, double dy, double dz, double r,
                                 int use_dir)
{
    double gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (!use_dir || gn == 0.0) return 1.0;
    double wix = dx / r, wiy = dy / r, wiz = dz / r;          /* incoming direction */
    double nx = gx / gn, ny = gy / gn, nz = gz / gn;          /* unit normal        */
    double nd = nx * wix + ny * wiy + nz * wiz;
    double wox = wix - 2.0 * nd * nx;                          /* ideal specular     */
    double woy = wiy - 2.0 * nd * ny;
    double woz = wiz - 2.0 * nd * nz;
    double wrx = -wix, wry = -wiy, wrz = -wiz;                 /* back to receiver   */
    double d = wox * wrx + woy * wry + woz * wrz;
    return d > 0.0 ? d : 0.0;
}

/* Lensless transmittance seen from antenna i (section 6, Eq. lens-less-
 * transmittance, integrated as in App. B.2): t_eff_j = T_j + Phi_s(f(x_apr)) is
 * the primary-ray transmittance plus the primary origin's sigmoid-SDF, c_ant_i
 * = Phi_s(f(a_i)) the real origin's; the result is clamped to [0, 1]. The
 * clamp's slope (the subgradient taken at its two kinks) is 1 on the closed
 * interval 0 <= t_eff - c_ant <= 1, decided in FP64 on the exact difference. */
static double lensless_T(double t_eff, double c_ant, int* inside)
{
    double v = t_eff - c_ant;
    *inside = (v >= 0.0 && v <= 1.0);
    if (v < 0.0) return 0.0;
    if (v > 1.0) return 1.0;
    return v;
}

/*
 * Signal tracing forward (section 5.1, Eq. ref_sim; App. A.6, Algorithm 2 [1]):
 *   s(i, n) = sum_j A_ij exp(-j phi_ijn),
 *   A_ij = w_j * T'_ij^2 * gamma_ij * D_ij      (section 5.2, Eq. signal_amp_tracing)
 * with w_j = a_j alpha_j A'_tx (blend output), T'_ij the lensless transmittance,
 * gamma_ij = 1 / (4 pi r_ij)^2 (section 3, Eq. reflection_angle; App. A.2) and
 * D_ij the directional factor. Parallel over antennas, serial over points.
 */
void oracle_render(long n_pts, const double* px, const double* py, const double* pz,
                   const double* gx, const double* gy, const double* gz,
                   const double* w, const double* t_eff,
                   long n_ant, const double* ax, const double* ay, const double* az,
                   const double* c_ant, double f0, double df, long n_f, int use_dir,
                   double* s_re, double* s_im)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < n_ant; ++i) {
        for (long n = 0; n < n_f; ++n) { s_re[i * n_f + n] = 0.0; s_im[i * n_f + n] = 0.0; }
        for (long j = 0; j < n_pts; ++j) {
            double dx = px[j] - ax[i], dy = py[j] - ay[i], dz = pz[j] - az[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            int inside;
            double t = lensless_T(t_eff[j], c_ant[i], &inside);
            double gamma = 1.0 / ((4.0 * M_PI * r) * (4.0 * M_PI * r));
            double D = directional_factor(gx[j], gy[j], gz[j], dx, dy, dz, r, use_dir);
            double A = w[j] * t * t * gamma * D;
            double tau = 2.0 * r / C_LIGHT;
            for (long n = 0; n < n_f; ++n) {
                double phi = TWO_PI * (f0 + (double)n * df) * tau;
                s_re[i * n_f + n] += A * cos(phi);
                s_im[i * n_f + n] -= A * sin(phi);
            }
        }
    }
}

/*
 * Signal tracing backward (App. A.5, gradient of Eq. ref_sim; Algorithm 2 [2]).
 * g = dL/dRe s + j dL/dIm s. For the real amplitude A_ij the derivative is
 *   q_ij = dL/dA_ij = sum_n Re( conj(g_in) exp(-j phi_ijn) ),
 * the real part the printed complex sum leaves implicit. The chain rule through
 * A_ij = w T'^2 gamma D then gives dL/dw_j, dL/dt_eff_j and dL/dG_j (G = grad f,
 * the unnormalised SDF gradient whose direction is the normal). Parallel over
 * points, serial over antennas and frequencies.
 */
void oracle_render_backward(long n_pts, const double* px, const double* py, const double* pz,
                            const double* gx, const double* gy, const double* gz,
                            const double* w, const double* t_eff,
                            long n_ant, const double* ax, const double* ay, const double* az,
                            const double* c_ant, double f0, double df, long n_f, int use_dir,
                            const double* g_re, const double* g_im,
                            double* d_w, double* d_teff, double* d_gx, double* d_gy, double* d_gz)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (long j = 0; j < n_pts; ++j) {
        double acc_w = 0.0, acc_t = 0.0, acc_gx = 0.0, acc_gy = 0.0, acc_gz = 0.0;
        double gn = sqrt(gx[j] * gx[j] + gy[j] * gy[j] + gz[j] * gz[j]);
        for (long i = 0; i < n_ant; ++i) {
            double dx = px[j] - ax[i], dy = py[j] - ay[i], dz = pz[j] - az[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            int inside;
            double t = lensless_T(t_eff[j], c_ant[i], &inside);
            double gamma = 1.0 / ((4.0 * M_PI * r) * (4.0 * M_PI * r));
            double D = directional_factor(gx[j], gy[j], gz[j], dx, dy, dz, r, use_dir);
            double tau = 2.0 * r / C_LIGHT;
            double q = 0.0;
            for (long n = 0; n < n_f; ++n) {
                double phi = TWO_PI * (f0 + (double)n * df) * tau;
                /* Re( (g_r - j g_i) (cos phi - j sin phi) ) */
                q += g_re[i * n_f + n] * cos(phi) - g_im[i * n_f + n] * sin(phi);
            }
            acc_w += t * t * gamma * D * q;
            if (inside) acc_t += w[j] * 2.0 * t * gamma * D * q;
            if (use_dir && gn > 0.0) {
                /* D = 2 c^2 - 1 with c = n.w_i, n = G/|G|; dD/dG = 4 c (w_i - c n) / |G| */
                double nx = gx[j] / gn, ny = gy[j] / gn, nz = gz[j] / gn;
                double wix = dx / r, wiy = dy / r, wiz = dz / r;
                double c = nx * wix + ny * wiy + nz * wiz;
                if (2.0 * c * c - 1.0 > 0.0) {
                    double k = w[j] * t * t * gamma * q * 4.0 * c / gn;
                    acc_gx += k * (wix - c * nx);
                    acc_gy += k * (wiy - c * ny);
                    acc_gz += k * (wiz - c * nz);
                }
            }
        }
        d_w[j] = acc_w; d_teff[j] = acc_t;
        d_gx[j] = acc_gx; d_gy[j] = acc_gy; d_gz[j] = acc_gz;
    }
}

/*
 * Matched filter forward (section 3, Eq. mf-sm; App. A.5; Algorithm 1 [1]):
 *   M_v = sum_i sum_n s(i, n) exp(+j phi_ivn),   P_v = |M_v|.
 * Parallel over voxels, serial over antennas and frequencies.
 */
void oracle_filter(long n_vox, const double* vx, const double* vy, const double* vz,
                   long n_ant, const double* ax, const double* ay, const double* az,
                   double f0, double df, long n_f,
                   const double* s_re, const double* s_im,
                   double* M_re, double* M_im, double* P)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (long v = 0; v < n_vox; ++v) {
        double mr = 0.0, mi = 0.0;
        for (long i = 0; i < n_ant; ++i) {
            double dx = vx[v] - ax[i], dy = vy[v] - ay[i], dz = vz[v] - az[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double tau = 2.0 * r / C_LIGHT;
            for (long n = 0; n < n_f; ++n) {
                double phi = TWO_PI * (f0 + (double)n * df) * tau;
                double c = cos(phi), s = sin(phi);
                double sr = s_re[i * n_f + n], si = s_im[i * n_f + n];
                mr += sr * c - si * s;
                mi += sr * s + si * c;
            }
        }
        M_re[v] = mr; M_im[v] = mi; P[v] = sqrt(mr * mr + mi * mi);
    }
}

/*
 * Matched filter backward (App. A.5; Algorithm 1 [2]). The derivative of
 * P_v = |M_v| with respect to s(i, n), written g = dL/dRe s + j dL/dIm s, is
 *   g(i, n) = sum_v dL/dP_v * (M_v / |M_v|) * exp(-j phi_ivn);
 * the printed formula drops the M_v factor (it writes 1/P). A voxel with
 * |M_v| = 0 contributes nothing. Parallel over antennas, serial over voxels.
 */
void oracle_filter_backward(long n_vox, const double* vx, const double* vy, const double* vz,
                            long n_ant, const double* ax, const double* ay, const double* az,
                            double f0, double df, long n_f,
                            const double* M_re, const double* M_im, const double* dP,
                            double* g_re, double* g_im)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < n_ant; ++i) {
        for (long n = 0; n < n_f; ++n) { g_re[i * n_f + n] = 0.0; g_im[i * n_f + n] = 0.0; }
        for (long v = 0; v < n_vox; ++v) {
            double m = sqrt(M_re[v] * M_re[v] + M_im[v] * M_im[v]);
            if (m == 0.0) continue;
            double cr = dP[v] * M_re[v] / m, ci = dP[v] * M_im[v] / m;
            double dx = vx[v] - ax[i], dy = vy[v] - ay[i], dz = vz[v] - az[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double tau = 2.0 * r / C_LIGHT;
            for (long n = 0; n < n_f; ++n) {
                double phi = TWO_PI * (f0 + (double)n * df) * tau;
                double c = cos(phi), s = sin(phi);
                /* (cr + j ci)(cos phi - j sin phi) */
                g_re[i * n_f + n] += cr * c + ci * s;
                g_im[i * n_f + n] += ci * c - cr * s;
            }
        }
    }
}

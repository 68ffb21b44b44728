/*
 * ewald_oracle.c - FP64 oracle for the long-range half of the electrostatics
 * that ACEMD evaluates by particle-mesh Ewald (section "Molecular dynamics on
 * the GPU": PME on the GPU with the FFT library; section "Validation": a 64^3
 * grid).  Written as the Ewald sum's plain definition: the reciprocal-space
 * sum over reciprocal lattice vectors m = (mx/Lx, my/Ly, mz/Lz),
 *
 *   E_rec = ke/(2 pi V) sum_{m != 0} exp(-pi^2 m^2 / alpha^2) / m^2 |S(m)|^2,
 *   S(m)  = sum_j q_j exp(2 pi i m . r_j),
 *
 * its exact gradient and its strain derivative (virial), and the
 * Ewald-consistent corrections that go with a reciprocal sum over all pairs:
 * the self term -ke alpha/sqrt(pi) sum q^2 and, per excluded pair,
 * -ke q_i q_j erf(alpha r)/r (per scaled 1-4 pair the same times 1 - s14).
 *
 * TEST INFRASTRUCTURE ONLY (compiled into liboracle.so with nb_oracle.c); it
 * shares no code with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Direct reciprocal-space Ewald sum over |m_a| <= k_a (integer components).
 * F [n*3] receives the forces, E[0] the energy, W[6] the virial
 * (xx, yy, zz, xy, xz, yz: W_ab = sum_m E(m) (delta_ab - 2 (1 + pi^2 m^2 /
 * alpha^2) m_a m_b / m^2)).  Returns 0, or -1 on allocation failure. */
int orc_ewald_recip(int64_t n, const float *pos, const float *q, const float *box, double alpha, double ke,
                    int kx, int ky, int kz, double *F, double *E, double *W)
{
    const double L[3] = {box[0], box[1], box[2]};
    const double V = L[0] * L[1] * L[2];
    const int K[3] = {kx, ky, kz};
    const int nm[3] = {2 * kx + 1, 2 * ky + 1, 2 * kz + 1};
    const int64_t nvec = (int64_t)nm[0] * nm[1] * nm[2];
    /* per atom and axis: exp(2 pi i m x / L) for m = -k..k */
    double *ere[3], *eim[3];
    for (int a = 0; a < 3; ++a) {
        ere[a] = malloc(sizeof(double) * n * nm[a]);
        eim[a] = malloc(sizeof(double) * n * nm[a]);
        if (!ere[a] || !eim[a]) return -1;
    }
    for (int a = 0; a < 3; ++a) {
#pragma omp parallel for
        for (int64_t i = 0; i < n; ++i) {
            const double t = 2.0 * M_PI * (double)pos[3 * i + a] / L[a];
            for (int m = -K[a]; m <= K[a]; ++m) {
                ere[a][i * nm[a] + m + K[a]] = cos(t * m);
                eim[a][i * nm[a] + m + K[a]] = sin(t * m);
            }
        }
    }
    double *Sre = calloc(nvec, sizeof(double)), *Sim = calloc(nvec, sizeof(double));
    double *g = calloc(nvec, sizeof(double));
    if (!Sre || !Sim || !g) return -1;
    double e = 0.0, w[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel for reduction(+ : e, w[:6]) schedule(dynamic, 16)
    for (int64_t v = 0; v < nvec; ++v) {
        const int mx = (int)(v / ((int64_t)nm[1] * nm[2])) - kx;
        const int my = (int)((v / nm[2]) % nm[1]) - ky;
        const int mz = (int)(v % nm[2]) - kz;
        if (mx == 0 && my == 0 && mz == 0) continue;
        const double m[3] = {mx / L[0], my / L[1], mz / L[2]};
        const double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double xr = ere[0][j * nm[0] + mx + kx], xi = eim[0][j * nm[0] + mx + kx];
            const double yr = ere[1][j * nm[1] + my + ky], yi = eim[1][j * nm[1] + my + ky];
            const double zr = ere[2][j * nm[2] + mz + kz], zi = eim[2][j * nm[2] + mz + kz];
            const double pr = xr * yr - xi * yi, pi_ = xr * yi + xi * yr;
            sr += q[j] * (pr * zr - pi_ * zi);
            si += q[j] * (pr * zi + pi_ * zr);
        }
        Sre[v] = sr;
        Sim[v] = si;
        g[v] = exp(-M_PI * M_PI * m2 / (alpha * alpha)) / m2;
        const double em = ke / (2.0 * M_PI * V) * g[v] * (sr * sr + si * si);
        e += em;
        const double c = 2.0 * (1.0 + M_PI * M_PI * m2 / (alpha * alpha)) / m2;
        w[0] += em * (1.0 - c * m[0] * m[0]);
        w[1] += em * (1.0 - c * m[1] * m[1]);
        w[2] += em * (1.0 - c * m[2] * m[2]);
        w[3] += em * (-c * m[0] * m[1]);
        w[4] += em * (-c * m[0] * m[2]);
        w[5] += em * (-c * m[1] * m[2]);
    }
    /* F_i = (2 ke q_i / V) sum_m g(m) m Im(conj(S(m)) exp(2 pi i m . r_i)) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double f[3] = {0, 0, 0};
        for (int64_t v = 0; v < nvec; ++v) {
            if (g[v] == 0.0) continue;
            const int mx = (int)(v / ((int64_t)nm[1] * nm[2])) - kx;
            const int my = (int)((v / nm[2]) % nm[1]) - ky;
            const int mz = (int)(v % nm[2]) - kz;
            const double xr = ere[0][i * nm[0] + mx + kx], xi = eim[0][i * nm[0] + mx + kx];
            const double yr = ere[1][i * nm[1] + my + ky], yi = eim[1][i * nm[1] + my + ky];
            const double zr = ere[2][i * nm[2] + mz + kz], zi = eim[2][i * nm[2] + mz + kz];
            const double pr = xr * yr - xi * yi, pi_ = xr * yi + xi * yr;
            const double er = pr * zr - pi_ * zi, ei = pr * zi + pi_ * zr;
            const double im = Sre[v] * ei - Sim[v] * er; /* Im(conj(S) e) */
            f[0] += g[v] * (mx / L[0]) * im;
            f[1] += g[v] * (my / L[1]) * im;
            f[2] += g[v] * (mz / L[2]) * im;
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = 2.0 * ke * (double)q[i] / V * f[a];
    }
    E[0] = e;
    for (int k = 0; k < 6; ++k) W[k] = w[k];
    for (int a = 0; a < 3; ++a) {
        free(ere[a]);
        free(eim[a]);
    }
    free(Sre);
    free(Sim);
    free(g);
    return 0;
}

/* Ewald-consistent corrections for a reciprocal sum over all pairs: the self
 * energy E[0] = -ke alpha/sqrt(pi) sum q^2, and E[1] = sum over excluded
 * pairs of -ke q_i q_j erf(alpha r)/r plus, over 1-4 pairs, (1 - s14c) times
 * the same; F [n*3] and W[6] receive the pair terms' forces and virial
 * (W_ab = sum d_ij,a f_ij,b, d_ij = x_i - x_j minimum image in FP64). */
void orc_ewald_corrections(int64_t n, const float *pos, const float *q, const float *box, double alpha, double ke,
                           int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14, double s14c, double *F,
                           double *E, double *W)
{
    const double L[3] = {box[0], box[1], box[2]};
    double qq = 0.0;
    for (int64_t i = 0; i < n; ++i) qq += (double)q[i] * q[i];
    E[0] = -ke * alpha / sqrt(M_PI) * qq;
    E[1] = 0.0;
    memset(F, 0, sizeof(double) * 3 * n);
    for (int k = 0; k < 6; ++k) W[k] = 0.0;
    for (int64_t p = 0; p < nex + n14; ++p) {
        const int32_t *pr = p < nex ? ex + 2 * p : p14 + 2 * (p - nex);
        const double wgt = p < nex ? 1.0 : 1.0 - s14c;
        const int64_t i = pr[0], j = pr[1];
        double d[3], r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double s = (double)pos[3 * i + a] - (double)pos[3 * j + a]; /* x_i - x_j */
            s -= L[a] * nearbyint(s / L[a]);
            d[a] = s;
            r2 += s * s;
        }
        const double r = sqrt(r2);
        const double c = wgt * ke * (double)q[i] * q[j];
        E[1] += -c * erf(alpha * r) / r;
        /* U = -c erf(a r)/r; dU/dr = -c (2a/sqrt(pi) exp(-a^2 r^2) r - erf(a r)) / r^2 */
        const double dudr = -c * (2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * r2) * r - erf(alpha * r)) / r2;
        for (int a = 0; a < 3; ++a) {
            const double f = -dudr * d[a] / r; /* force on i */
            F[3 * i + a] += f;
            F[3 * j + a] -= f;
        }
        const double fs = -dudr / r;
        W[0] += d[0] * fs * d[0];
        W[1] += d[1] * fs * d[1];
        W[2] += d[2] * fs * d[2];
        W[3] += d[0] * fs * d[1];
        W[4] += d[0] * fs * d[2];
        W[5] += d[1] * fs * d[2];
    }
}

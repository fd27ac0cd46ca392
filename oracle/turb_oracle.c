/*
 * turb_oracle.c -- plain, slow, FP64 CPU oracle for the split-step turbulence path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  The CUDA library never links, includes or calls it, and it shares no
 * code, header, table or constant generator with the CUDA kernels.
 *
 * Everything is double precision and follows the paper (TurPy, arXiv 2604.07248) step by step in
 * its own notation.  Nothing is blocked, fused or reordered beyond what the definitions state; the
 * only "library-like" piece is the textbook iterative radix-2 FFT below, written here from its
 * definition.
 *
 * Conventions (readings of the paper where it is silent or garbled):
 *   - FFT2 is the unnormalised forward DFT  X[k] = sum_n x[n] exp(-2 pi i n k / N);
 *     IFFT2 carries the 1/N^2 (propagation, Eq. 1).  Screens use the unnormalised inverse sum
 *     (Eq. S16), i.e. N^2 * ifft2.
 *   - Spectral index map f(n) = n for n < N/2, else n - N; kappa = (2 pi / (N dx)) * f(n).
 *   - Complex Gaussian noise N_c(0,1): real and imaginary parts each N(0,1) (Eq. 2, S16).
 *   - The phase PSD is Phi_phi = 2 pi k^2 dz * 0.033 Cn^2 (kappa^2 + kappa0^2)^(-11/6)
 *     exp(-kappa^2/kappa_m^2), kappa0 = 2 pi / L0, kappa_m = 2 pi / l0 (S14, S17, S18, angular);
 *     other media of Table S1 replace 11/3 by their power law alpha and 0.033 by a constant A.
 *   - H = exp(-i dz kappa^2 / (k + sqrt(k^2 - kappa^2))) = H_as * exp(-i k dz)  (Sec. 2.4; the
 *     global piston exp(i k dz) is dropped), 0 in the evanescent region.
 *
 * Parity status of each function is stated in its comment; all are pinned by the CPU tests except
 * where the comment says "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",   */
/* SC'11.  Ten rounds of the 4x32 Philox S-box with Weyl key schedule.                          */
/* Pinned by the published known-answer vectors (tests/golden/philox4x32_10_kat.txt).          */
/* ------------------------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* u32 word -> uniform in (0,1): ((w >> 8) + 0.5) * 2^-24, exact in binary32 and binary64. */
static double u01(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Box-Muller (Box & Muller 1958): two uniforms -> one complex sample with independent N(0,1)
 * real and imaginary parts. */
static cplx box_muller(uint32_t wa, uint32_t wb)
{
    double ua = u01(wa), ub = u01(wb);
    double rad = sqrt(-2.0 * log(ua));
    double ang = 2.0 * M_PI * ub;
    return rad * cos(ang) + I * (rad * sin(ang));
}

/* Counter layout (a choice of this project; the paper only asks for N_c(0,1), Eq. 2 / S16):
 *   key  = (seed mod 2^32, seed >> 32)
 *   ctr  = (word0, screen s, realization r, (purpose << 24) | t)
 * Grid noise (purpose 0): bins (m, n) and (m + N/2, n), m < N/2, share word0 = m N + n; the first
 * takes words (0,1), the second words (2,3).
 * Subharmonic noise (purpose 1): level p (1..3), sub-grid cell q = (m'+1)*3 + (n'+1) takes
 * word0 = (p-1)*8 + q/2, words (0,1) for even q and (2,3) for odd q. */
cplx orc_noise_bin(int N, uint64_t seed, uint32_t s, uint32_t r, uint32_t t, int m, int n)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int half = N / 2;
    int mm = m < half ? m : m - half;
    uint32_t ctr[4] = {(uint32_t)(mm * N + n), s, r, t & 0xFFFFFFu};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return m < half ? box_muller(w[0], w[1]) : box_muller(w[2], w[3]);
}

void orc_noise_grid(int N, uint64_t seed, uint32_t s, uint32_t r, uint32_t t, double* c_out)
{
    cplx* c = (cplx*)c_out;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) c[(size_t)m * N + n] = orc_noise_bin(N, seed, s, r, t, m, n);
}

cplx orc_noise_sh(uint64_t seed, uint32_t s, uint32_t r, uint32_t t, int p, int q)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)((p - 1) * 8 + q / 2), s, r, (1u << 24) | (t & 0xFFFFFFu)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return (q % 2 == 0) ? box_muller(w[0], w[1]) : box_muller(w[2], w[3]);
}

/* Raw export of the noise for tests: c_out holds 9 complex per level for levels 1..3. */
void orc_noise_sh_all(uint64_t seed, uint32_t s, uint32_t r, uint32_t t, double* c_out)
{
    cplx* c = (cplx*)c_out;
    for (int p = 1; p <= 3; ++p)
        for (int q = 0; q < 9; ++q) c[(p - 1) * 9 + q] = orc_noise_sh(seed, s, r, t, p, q);
}

/* ------------------------------------------------------------------------------------------ */
/* DFT.  Iterative radix-2 Cooley-Tukey (decimation in time), in place, unnormalised.            */
/* sign = -1: forward, exp(-2 pi i n k / N);  sign = +1: inverse sum, exp(+2 pi i n k / N).      */
/* Pinned against the brute-force DFT sum and against numpy.fft in the tests.                    */
/* ------------------------------------------------------------------------------------------ */
void orc_fft(int n, double* data, int sign)
{
    cplx* x = (cplx*)data;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx tmp = x[i];
            x[i] = x[j];
            x[j] = tmp;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int h = len / 2;
        for (int k = 0; k < h; ++k) {
            double ang = sign * 2.0 * M_PI * (double)k / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (int start = 0; start < n; start += len) {
                cplx a = x[start + k];
                cplx b = w * x[start + k + h];
                x[start + k] = a + b;
                x[start + k + h] = a - b;
            }
        }
    }
}

/* 2-D DFT of a row-major N x N array: all rows, then all columns (unnormalised). */
void orc_fft2(int N, double* data, int sign)
{
    cplx* x = (cplx*)data;
    cplx* col = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    for (int j = 0; j < N; ++j) orc_fft(N, (double*)(x + (size_t)j * N), sign);
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < N; ++j) col[j] = x[(size_t)j * N + i];
        orc_fft(N, (double*)col, sign);
        for (int j = 0; j < N; ++j) x[(size_t)j * N + i] = col[j];
    }
    free(col);
}

/* ------------------------------------------------------------------------------------------ */
/* Medium and grid.                                                                              */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double lambda; /* vacuum wavelength [m] */
    double n0;     /* mean refractive index */
    double l0;     /* inner scale [m]; <= 0 -> no inner-scale roll-off */
    double L0;     /* outer scale [m]; <= 0 or inf -> no outer scale */
    int N;         /* grid size (power of two) */
    double dx;     /* grid spacing [m] */
    double alpha;  /* power law of the index PSD, Phi_n ~ kappa^-alpha (Table S1); <= 0 -> 11/3 */
    double A;      /* constant of the index PSD; <= 0 -> 0.033 (Kolmogorov, S17 with S18) */
} orc_medium;

static double kspace(int N, int n) { return (double)(n < N / 2 ? n : n - N); }
static double dkappa(const orc_medium* md) { return 2.0 * M_PI / ((double)md->N * md->dx); }
static double wavenumber(const orc_medium* md) { return 2.0 * M_PI * md->n0 / md->lambda; }

/* Modified von Karman refractive-index PSD, S17 with kappa_m = 2 pi / l0 and kappa0 = 2 pi / L0,
 * written through Cn^2 (S18): Phi_n = 0.033 Cn^2 (kappa^2 + kappa0^2)^(-11/6) exp(-kappa^2/kappa_m^2).
 * For another medium of Table S1 the power law is Phi_n ~ kappa^-alpha (S12), alpha = beta + 3
 * (S11), with the same inner / outer-scale modification:
 *   Phi_n = A Cn^2 (kappa^2 + kappa0^2)^(-alpha/2) exp(-kappa^2/kappa_m^2).
 * The paper gives the law up to its constant; A is the caller's (orc_power_law_constant gives the
 * one for which Cn^2 is the index structure constant, D_n(r) = Cn^2 r^(alpha-3)). */
static double psd_alpha(const orc_medium* md) { return md->alpha > 0.0 ? md->alpha : 11.0 / 3.0; }
static double psd_const(const orc_medium* md) { return md->A > 0.0 ? md->A : 0.033; }

static double phi_n(const orc_medium* md, double cn2, double kappa2)
{
    double k0sq = (md->L0 > 0.0 && isfinite(md->L0)) ? pow(2.0 * M_PI / md->L0, 2.0) : 0.0;
    double kmsq = md->l0 > 0.0 ? pow(2.0 * M_PI / md->l0, 2.0) : INFINITY;
    double roll = isinf(kmsq) ? 1.0 : exp(-kappa2 / kmsq);
    return psd_const(md) * cn2 * pow(kappa2 + k0sq, -psd_alpha(md) / 2.0) * roll;
}

/* The constant A(alpha) of a power-law index PSD A Cn^2 kappa^-alpha whose structure function is
 * D_n(r) = Cn^2 r^(alpha - 3) (3 < alpha < 5), where D_n(r) = 8 pi int (1 - sin(kappa r)/(kappa r))
 * Phi_n(kappa) kappa^2 dkappa: the published non-Kolmogorov constant
 *   A(alpha) = Gamma(alpha - 1) cos(pi alpha / 2) / (4 pi^2)
 * (Toselli, Andrews, Phillips, Ferrero 2007), 0.0330 at alpha = 11/3 (the Kolmogorov 0.033).  Pinned
 * in the tests against the defining integral, evaluated numerically. */
double orc_power_law_constant(double alpha)
{
    return tgamma(alpha - 1.0) * cos(M_PI * alpha / 2.0) / (4.0 * M_PI * M_PI);
}

/* Phase PSD of one screen covering an interval dz: S14, Phi_phi = 2 pi k^2 dz Phi_n. */
double orc_phase_psd(const orc_medium* md, double cn2, double dz, double kappa2)
{
    double k = wavenumber(md);
    return 2.0 * M_PI * k * k * dz * phi_n(md, cn2, kappa2);
}

/* Spectral amplitude s(kappa) = sqrt(Phi_phi dkx dky) on the N x N grid (Eq. S16), s(0,0) = 0. */
void orc_psd_amplitude(const orc_medium* md, double cn2, double dz, double* s_out)
{
    int N = md->N;
    double dk = dkappa(md);
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) {
            double kx = dk * kspace(N, n), ky = dk * kspace(N, m);
            double kap2 = kx * kx + ky * ky;
            s_out[(size_t)m * N + n] = (m == 0 && n == 0) ? 0.0 : sqrt(orc_phase_psd(md, cn2, dz, kap2)) * dk;
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Subharmonics, Eq. 2: levels p = 1..3, scale s = 3, 3x3 sub-grid per level without (0,0).     */
/* Coefficient a[p][q] = sqrt(Phi_phi(kappa_pq)) (dk / 3^p) c[p][q], kappa_pq = (n', m') dk / 3^p */
/* with q = (m'+1)*3 + (n'+1).                                                                   */
/* ------------------------------------------------------------------------------------------ */
void orc_sh_amplitude(const orc_medium* md, double cn2, double dz, double* b_out /* 27 */)
{
    double dk = dkappa(md);
    for (int p = 1; p <= 3; ++p) {
        double dkp = dk / pow(3.0, p);
        for (int q = 0; q < 9; ++q) {
            int mp = q / 3 - 1, np = q % 3 - 1;
            double kx = np * dkp, ky = mp * dkp;
            b_out[(p - 1) * 9 + q] = (mp == 0 && np == 0) ? 0.0 : sqrt(orc_phase_psd(md, cn2, dz, kx * kx + ky * ky)) * dkp;
        }
    }
}

/* phi_SH[j,i] = sum_p sum_q Re(a[p][q] exp(i (kx x + ky y))), x = i dx, y = j dx (Eq. 2),
 * evaluated term by term at every pixel. */
void orc_sh_screen(const orc_medium* md, const double* a_in /* 27 complex */, double* phi_sh)
{
    const cplx* a = (const cplx*)a_in;
    int N = md->N;
    double dk = dkappa(md);
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double x = i * md->dx, y = j * md->dx, acc = 0.0;
            for (int p = 1; p <= 3; ++p) {
                double dkp = dk / pow(3.0, p);
                for (int q = 0; q < 9; ++q) {
                    int mp = q / 3 - 1, np = q % 3 - 1;
                    if (mp == 0 && np == 0) continue;
                    double arg = np * dkp * x + mp * dkp * y;
                    acc += creal(a[(p - 1) * 9 + q] * (cos(arg) + I * sin(arg)));
                }
            }
            phi_sh[(size_t)j * N + i] = acc;
        }
}

/* Screen from its spectrum: phi = Re(unnormalised inverse DFT(spec)) (S16) + phi_SH (Eq. 3),
 * minus the mean of the sum (piston removal, after S16).  sh may be NULL (no subharmonics). */
void orc_screen_from_spectrum(const orc_medium* md, const double* spec_in, const double* sh, double* phi)
{
    int N = md->N;
    size_t N2 = (size_t)N * N;
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * N2);
    memcpy(tmp, spec_in, sizeof(cplx) * N2);
    orc_fft2(N, (double*)tmp, +1);
    double* phsh = NULL;
    if (sh) {
        phsh = (double*)malloc(sizeof(double) * N2);
        orc_sh_screen(md, sh, phsh);
    }
    double mean = 0.0;
    for (size_t k = 0; k < N2; ++k) {
        phi[k] = creal(tmp[k]) + (phsh ? phsh[k] : 0.0);
        mean += phi[k];
    }
    mean /= (double)N2;
    for (size_t k = 0; k < N2; ++k) phi[k] -= mean;
    free(phsh);
    free(tmp);
}

/* Initial (t = 0) spectrum and subharmonic coefficients of screen s, realization r:
 * spec = s(kappa) * c^(0) (S16), a = b * c_SH^(0) (Eq. 2).  sh_levels is 0 or 3. */
void orc_screen_spectrum(const orc_medium* md, double cn2, double dz, int sh_levels, uint64_t seed, uint32_t s,
                         uint32_t r, uint32_t t, double* spec_out, double* sh_out)
{
    int N = md->N;
    size_t N2 = (size_t)N * N;
    double* amp = (double*)malloc(sizeof(double) * N2);
    orc_psd_amplitude(md, cn2, dz, amp);
    cplx* spec = (cplx*)spec_out;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) spec[(size_t)m * N + n] = amp[(size_t)m * N + n] * orc_noise_bin(N, seed, s, r, t, m, n);
    free(amp);
    if (sh_levels > 0 && sh_out) {
        double b[27];
        orc_sh_amplitude(md, cn2, dz, b);
        cplx* a = (cplx*)sh_out;
        for (int p = 1; p <= 3; ++p)
            for (int q = 0; q < 9; ++q) a[(p - 1) * 9 + q] = b[(p - 1) * 9 + q] * orc_noise_sh(seed, s, r, t, p, q);
    }
}

/* One independent screen (Fig. 1B-C, S16, Eq. 2-3). */
void orc_make_screen(const orc_medium* md, double cn2, double dz, int sh_levels, uint64_t seed, uint32_t s,
                     uint32_t r, double* phi)
{
    size_t N2 = (size_t)md->N * md->N;
    double* spec = (double*)malloc(sizeof(double) * 2 * N2);
    double sh[54];
    orc_screen_spectrum(md, cn2, dz, sh_levels, seed, s, r, 0, spec, sh);
    orc_screen_from_spectrum(md, spec, sh_levels > 0 ? sh : NULL, phi);
    free(spec);
}

/* ------------------------------------------------------------------------------------------ */
/* AR(1) evolution, Eq. 4-5 (Sec. 2.3):                                                           */
/*   spec_t = alpha * exp(i theta) * spec_{t-1} + sqrt(1 - alpha^2) * s(kappa) * c^(t),          */
/*   theta  = -2 pi T (fx vx + fy vy),  f = kappa / (2 pi)  (Eq. 4, with the lost i restored).   */
/* The 24 subharmonic coefficients follow the same rule with their own (sub-grid) frequencies.    */
/* ------------------------------------------------------------------------------------------ */
void orc_ar_step(const orc_medium* md, double cn2, double dz, int sh_levels, uint64_t seed, uint32_t s, uint32_t r,
                 uint32_t t, double alpha, double vx, double vy, double T, double* spec_io, double* sh_io)
{
    int N = md->N;
    double dk = dkappa(md);
    double beta = sqrt(1.0 - alpha * alpha);
    size_t N2 = (size_t)N * N;
    double* amp = (double*)malloc(sizeof(double) * N2);
    orc_psd_amplitude(md, cn2, dz, amp);
    cplx* spec = (cplx*)spec_io;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) {
            double fx = dk * kspace(N, n) / (2.0 * M_PI), fy = dk * kspace(N, m) / (2.0 * M_PI);
            double theta = -2.0 * M_PI * T * (fx * vx + fy * vy);
            cplx tilt = cos(theta) + I * sin(theta);
            size_t k = (size_t)m * N + n;
            spec[k] = alpha * tilt * spec[k] + beta * amp[k] * orc_noise_bin(N, seed, s, r, t, m, n);
        }
    free(amp);
    if (sh_levels > 0 && sh_io) {
        double b[27];
        orc_sh_amplitude(md, cn2, dz, b);
        cplx* a = (cplx*)sh_io;
        for (int p = 1; p <= 3; ++p) {
            double dkp = dk / pow(3.0, p);
            for (int q = 0; q < 9; ++q) {
                int mp = q / 3 - 1, np = q % 3 - 1;
                double fx = np * dkp / (2.0 * M_PI), fy = mp * dkp / (2.0 * M_PI);
                double theta = -2.0 * M_PI * T * (fx * vx + fy * vy);
                cplx tilt = cos(theta) + I * sin(theta);
                int k = (p - 1) * 9 + q;
                a[k] = alpha * tilt * a[k] + beta * b[k] * orc_noise_sh(seed, s, r, t, p, q);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Sources (S22; plane wave of Sec. 3.3), centred on pixel (N/2, N/2).                            */
/* ------------------------------------------------------------------------------------------ */
void orc_source_gaussian(int N, double dx, double w0, double* U_out)
{
    cplx* U = (cplx*)U_out;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double x = (i - N / 2) * dx, y = (j - N / 2) * dx;
            U[(size_t)j * N + i] = exp(-(x * x + y * y) / (w0 * w0));
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Angular-spectrum transfer function without its piston (Sec. 2.4):                              */
/*   H = exp(-i dz kappa^2 / (k + sqrt(k^2 - kappa^2)))  for kappa^2 < k^2, else 0.               */
/* (dz (sqrt(k^2 - kappa^2) - k) rewritten without the cancellation.)                             */
/* ------------------------------------------------------------------------------------------ */
void orc_transfer(const orc_medium* md, double dz, double* H_out)
{
    int N = md->N;
    double dk = dkappa(md), k = wavenumber(md);
    cplx* H = (cplx*)H_out;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) {
            double kx = dk * kspace(N, n), ky = dk * kspace(N, m);
            double kap2 = kx * kx + ky * ky;
            cplx h = 0.0;
            if (kap2 < k * k) {
                double ph = -dz * kap2 / (k + sqrt(k * k - kap2));
                h = cos(ph) + I * sin(ph);
            }
            H[(size_t)m * N + n] = h;
        }
}

/* Split-step propagation, Eq. 1, for s = 1..S:  U <- IFFT2(FFT2(U) * H_s) * exp(i phi_s).
 * phi holds S screens (N x N each); a NULL phi means vacuum (no modulation). */
void orc_propagate(const orc_medium* md, int S, const double* dz, const double* phi, double* U_io)
{
    int N = md->N;
    size_t N2 = (size_t)N * N;
    cplx* U = (cplx*)U_io;
    cplx* H = (cplx*)malloc(sizeof(cplx) * N2);
    for (int s = 0; s < S; ++s) {
        orc_transfer(md, dz[s], (double*)H);
        orc_fft2(N, U_io, -1);
        for (size_t k = 0; k < N2; ++k) U[k] *= H[k];
        orc_fft2(N, U_io, +1);
        for (size_t k = 0; k < N2; ++k) U[k] /= (double)N2;
        if (phi) {
            const double* ph = phi + (size_t)s * N2;
            for (size_t k = 0; k < N2; ++k) U[k] *= cos(ph[k]) + I * sin(ph[k]);
        }
    }
    free(H);
}

/* Adjoint of orc_propagate with respect to the complex field (gradient convention
 * g = dL/dRe + i dL/dIm, so a linear map P back-propagates as P^H).  For s = S..1:
 *   g <- g * exp(-i phi_s);  g <- IFFT2(FFT2(g) * conj(H_s)). */
void orc_propagate_adjoint(const orc_medium* md, int S, const double* dz, const double* phi, double* g_io)
{
    int N = md->N;
    size_t N2 = (size_t)N * N;
    cplx* g = (cplx*)g_io;
    cplx* H = (cplx*)malloc(sizeof(cplx) * N2);
    for (int s = S - 1; s >= 0; --s) {
        if (phi) {
            const double* ph = phi + (size_t)s * N2;
            for (size_t k = 0; k < N2; ++k) g[k] *= cos(ph[k]) - I * sin(ph[k]);
        }
        orc_transfer(md, dz[s], (double*)H);
        orc_fft2(N, g_io, -1);
        for (size_t k = 0; k < N2; ++k) g[k] *= conj(H[k]);
        orc_fft2(N, g_io, +1);
        for (size_t k = 0; k < N2; ++k) g[k] /= (double)N2;
    }
    free(H);
}

/* ------------------------------------------------------------------------------------------ */
/* Moments (S25 with Welford's update, Sec. 3.3; second-moment radius, Sec. 3.2).               */
/* ------------------------------------------------------------------------------------------ */
/* One Welford step per pixel for realization count n (after the update, n >= 1). */
void orc_welford_update(size_t npix, const double* I_in, long n, double* mean, double* M2)
{
    for (size_t k = 0; k < npix; ++k) {
        double d = I_in[k] - mean[k];
        mean[k] += d / (double)n;
        M2[k] += d * (I_in[k] - mean[k]);
    }
}

/* Chan, Golub, LeVeque pairwise merge of (n_a, mean_a, M2_a) with (n_b, mean_b, M2_b) into a. */
void orc_welford_merge(size_t npix, long na, double* mean_a, double* M2_a, long nb, const double* mean_b,
                       const double* M2_b)
{
    double n = (double)(na + nb);
    for (size_t k = 0; k < npix; ++k) {
        double d = mean_b[k] - mean_a[k];
        mean_a[k] += d * (double)nb / n;
        M2_a[k] += M2_b[k] + d * d * (double)na * (double)nb / n;
    }
}

/* Per-realization sums of I and r^2 I, r measured from pixel (N/2, N/2). */
void orc_beam_sums(int N, double dx, const double* I_in, double* sumI, double* sumR2I)
{
    double a = 0.0, b = 0.0;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double x = (i - N / 2) * dx, y = (j - N / 2) * dx;
            double v = I_in[(size_t)j * N + i];
            a += v;
            b += (x * x + y * y) * v;
        }
    *sumI = a;
    *sumR2I = b;
}

/* ------------------------------------------------------------------------------------------ */
/* Dual-domain two-mask D2NN receiver (Sec. 2.5, 4.1).                                             */
/* C = fftshift o fft2 o ifftshift / N (unitary lens DFT), C^-1 = fftshift o ifft2 o ifftshift N. */
/* ------------------------------------------------------------------------------------------ */
static void roll_half(int N, cplx* x)
{
    /* for even N, fftshift == ifftshift == cyclic shift by N/2 in both axes */
    int h = N / 2;
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < N; ++i) {
            int i2 = (i + h) % N, j2 = j + h;
            cplx t = x[(size_t)j * N + i];
            x[(size_t)j * N + i] = x[(size_t)j2 * N + i2];
            x[(size_t)j2 * N + i2] = t;
        }
}

void orc_lens_dft(int N, double* x_io, int inverse)
{
    cplx* x = (cplx*)x_io;
    size_t N2 = (size_t)N * N;
    roll_half(N, x);
    orc_fft2(N, x_io, inverse ? +1 : -1);
    roll_half(N, x);
    for (size_t k = 0; k < N2; ++k) x[k] /= (double)N;
}

void orc_aperture(int N, double dx, double diameter, double* A)
{
    double r2max = 0.25 * diameter * diameter;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            double x = (i - N / 2) * dx, y = (j - N / 2) * dx;
            A[(size_t)j * N + i] = (x * x + y * y <= r2max) ? 1.0 : 0.0;
        }
}

/* Forward receiver for one field U (N x N complex):
 *   Z1 = exp(i th1) A U;  W1 = C(Z1);  W2 = exp(i th2) W1;  V = C^-1(W2);  I = |V|^2.
 * Writes I; also returns Z1, W2 and V when the pointers are not NULL (needed by the adjoint). */
void orc_d2nn_forward(int N, const double* A, const double* th1, const double* th2, const double* U_in, double* I_out,
                      double* Z1_out, double* W2_out, double* V_out)
{
    size_t N2 = (size_t)N * N;
    const cplx* U = (const cplx*)U_in;
    cplx* z = (cplx*)malloc(sizeof(cplx) * N2);
    for (size_t k = 0; k < N2; ++k) z[k] = A[k] * (cos(th1[k]) + I * sin(th1[k])) * U[k];
    if (Z1_out) memcpy(Z1_out, z, sizeof(cplx) * N2);
    orc_lens_dft(N, (double*)z, 0);
    for (size_t k = 0; k < N2; ++k) z[k] *= cos(th2[k]) + I * sin(th2[k]);
    if (W2_out) memcpy(W2_out, z, sizeof(cplx) * N2);
    orc_lens_dft(N, (double*)z, 1);
    if (V_out) memcpy(V_out, z, sizeof(cplx) * N2);
    for (size_t k = 0; k < N2; ++k) I_out[k] = creal(z[k]) * creal(z[k]) + cimag(z[k]) * cimag(z[k]);
    free(z);
}

/* Loss contribution of one field and dL/dI.  kind 0: MAE |I - I_ref| (Sec. 2.5); kind 1: squared
 * error.  Both are divided by `count` (the number of terms in the mean over batch and pixels). */
double orc_intensity_loss(size_t npix, const double* I_in, const double* Iref, int kind, double count, double* dLdI)
{
    double L = 0.0;
    for (size_t k = 0; k < npix; ++k) {
        double e = I_in[k] - Iref[k];
        if (kind == 0) {
            L += fabs(e);
            if (dLdI) dLdI[k] = (e > 0.0 ? 1.0 : (e < 0.0 ? -1.0 : 0.0)) / count;
        } else {
            L += e * e;
            if (dLdI) dLdI[k] = 2.0 * e / count;
        }
    }
    return L / count;
}

/* Adjoint of the receiver for one field: given dL/dI, accumulates dL/dth1 and dL/dth2 into
 * g_th1/g_th2 and writes g_U = dL/dU (complex, convention dL/dRe + i dL/dIm).
 *   g_V = 2 V dL/dI;  g_W2 = C(g_V);  dL/dth2 += Im(g_W2 conj(W2));
 *   g_W1 = exp(-i th2) g_W2;  g_Z1 = C^-1(g_W1);  dL/dth1 += Im(g_Z1 conj(Z1));
 *   g_U = A exp(-i th1) g_Z1. */
void orc_d2nn_backward(int N, const double* A, const double* th1, const double* th2, const double* Z1_in,
                       const double* W2_in, const double* V_in, const double* dLdI, double* g_th1, double* g_th2,
                       double* gU_out)
{
    size_t N2 = (size_t)N * N;
    const cplx* Z1 = (const cplx*)Z1_in;
    const cplx* W2 = (const cplx*)W2_in;
    const cplx* V = (const cplx*)V_in;
    cplx* g = (cplx*)malloc(sizeof(cplx) * N2);
    for (size_t k = 0; k < N2; ++k) g[k] = 2.0 * V[k] * dLdI[k];
    orc_lens_dft(N, (double*)g, 0);
    for (size_t k = 0; k < N2; ++k) {
        g_th2[k] += cimag(g[k] * conj(W2[k]));
        g[k] *= cos(th2[k]) - I * sin(th2[k]);
    }
    orc_lens_dft(N, (double*)g, 1);
    cplx* gU = (cplx*)gU_out;
    for (size_t k = 0; k < N2; ++k) {
        g_th1[k] += cimag(g[k] * conj(Z1[k]));
        gU[k] = A[k] * (cos(th1[k]) - I * sin(th1[k])) * g[k];
    }
    free(g);
}

/*
 * FP64 CPU oracle for the TACAW hot path (arXiv 2602.10064, PySlice).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load.  The CUDA library never
 * links, includes or calls it, and it shares no code, header or table with that library.
 *
 * It is the plain definition of the method, written for a reader to check by eye:
 *   - Methods, "Key Technical Elements", Multislice Propagation: transmission
 *     t = exp(i sigma V), Fresnel propagator P(k) = exp(-i pi lambda dz |k|^2), and the chain
 *     psi_exit = P t ... P t psi_probe (a transmission then a propagation per slice);
 *   - same section, Atomic Scattering Potentials: Kirkland's form factor
 *     f(q) = sum_i a_i/(q^2+b_i) + c_i exp(-d_i q^2), the slice potential assembled in
 *     reciprocal space as V(k) = sum_j f_Zj(k) exp(-2 pi i k.r_j) over the atoms inside the
 *     slice's z-bounds, then an inverse FFT;
 *   - Methods, "Workflow Architecture": psi~(k,w) = F_t[psi(k,t) - <psi(k,t)>_t] and the
 *     intensity I(k,w) = |psi~(k,w)|^2;
 *   - Supplement, "Sampling Considerations": dk = 1/L, df = 1/(N dt), f_max = 1/(2 dt).
 * Where the paper is silent the readings are:
 *   - prefactor 2 pi a0 e / A on V(k) with an unnormalised inverse DFT sum (V in V*A);
 *   - sigma = 2 pi gamma m0 e lambda / h^2 (relativistic mass; the paper drops e);
 *   - each atom wholly projected into the slice holding its centre; slice index from FP64
 *     z wrapped into [0, Lz) and floor(z / dz), dz = Lz / S, clamped to [0, S-1];
 *   - a circular 2/3 band limit |k|^2 <= kbl^2, kbl = frac * min(nx/(2Lx), ny/(2Ly)), applied
 *     to V(k), to the propagator in every slice and (optionally) to t;
 *   - unitary 2D FFTs for the wave: psi(k) = DFT(psi(r)) / sqrt(Nq);
 *   - plane wave psi0 = 1/sqrt(Nq); convergent probe psi0(k) = A(k) exp(-2 pi i k.r_p) / norm
 *     with A = 1 for |k| <= alpha/lambda, normalised to sum_k |psi0(k)|^2 = 1;
 *   - time transform with sign exp(-2 pi i m n / F), unnormalised, all F bins (fftfreq order).
 * The in-house FFT is a library-style primitive; the tests pin it to the O(N^2) DFT.
 * Parity of absolute physical intensity is unpinned: the form-factor table is an input and
 * the repository ships only a labelled synthetic placeholder table.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* CODATA 2018 values (h, e, c exact in SI). */
static const double O_H = 6.62607015e-34;     /* J s */
static const double O_QE = 1.602176634e-19;   /* C */
static const double O_ME = 9.1093837015e-31;  /* kg */
static const double O_C = 299792458.0;        /* m/s */
static const double O_A0 = 0.529177210903;    /* Bohr radius, A */
static const double O_EPS0 = 8.8541878128e-12;/* F/m */

typedef struct {
    int32_t nx, ny, n_slices;
    int32_t bandlimit_transmission; /* 1: t <- IDFT(M DFT(t)) / Nq */
    int32_t final_propagator;       /* 1: propagate after the last transmission */
    int32_t pad_;
    double Lx, Ly, Lz;              /* A */
    double voltage_ev;
    double bandlimit;               /* fraction of Nyquist; <= 0 switches every mask off */
    double sigma_scale;             /* multiplies sigma (1 = physical) */
} oracle_params;

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- electron optics ------------------------------------------------------------------ */

/* Relativistic electron wavelength in A: lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2))). */
double oracle_wavelength(double V) {
    double eV = O_QE * V;
    double p = sqrt(2.0 * O_ME * eV * (1.0 + eV / (2.0 * O_ME * O_C * O_C)));
    return O_H / p * 1e10;
}

/* Interaction parameter in rad/(V A): sigma = 2 pi m e lambda / h^2 with m = gamma m0. */
double oracle_sigma(double V) {
    double gamma = 1.0 + O_QE * V / (O_ME * O_C * O_C);
    double lam_m = oracle_wavelength(V) * 1e-10;
    return 2.0 * M_PI * gamma * O_ME * O_QE * lam_m / (O_H * O_H) * 1e-10;
}

/* 2 pi a0 e in V A^2, with e taken as e/(4 pi eps0) in V A. */
double oracle_kirkland_prefactor(void) {
    double e_VA = O_QE / (4.0 * M_PI * O_EPS0) * 1e10;
    return 2.0 * M_PI * O_A0 * e_VA;
}

/* Kirkland's form: coef = a1 b1 a2 b2 a3 b3 c1 d1 c2 d2 c3 d3; q in 1/A without 2 pi. */
double oracle_form_factor(const double *coef, double q) {
    double q2 = q * q, f = 0.0;
    for (int i = 0; i < 3; i++) f += coef[2 * i] / (q2 + coef[2 * i + 1]);
    for (int i = 0; i < 3; i++) f += coef[6 + 2 * i] * exp(-coef[7 + 2 * i] * q2);
    return f;
}

/* ---- grids ----------------------------------------------------------------------------- */

/* fftfreq: spatial frequency (cycles/A) of index i on an n-point axis of length L. */
double oracle_kfreq(int i, int n, double L) {
    int m = (i < (n + 1) / 2) ? i : i - n;
    return (double)m / L;
}

double oracle_kbl(const oracle_params *p) {
    double a = 0.5 * (double)p->nx / p->Lx, b = 0.5 * (double)p->ny / p->Ly;
    return p->bandlimit * (a < b ? a : b);
}

/* Band-limit mask, inclusive edge. */
int oracle_mask(const oracle_params *p, int iy, int ix) {
    if (p->bandlimit <= 0.0) return 1;
    double kx = oracle_kfreq(ix, p->nx, p->Lx), ky = oracle_kfreq(iy, p->ny, p->Ly);
    double k2 = kx * kx + ky * ky, kbl = oracle_kbl(p);
    return k2 <= kbl * kbl;
}

/* Slice index of height z (A): wrap into [0, Lz), floor(z/dz), clamp to [0, S-1]. */
int oracle_slice_index(double z, double Lz, int S) {
    double dz = Lz / (double)S;
    double zw = z - Lz * floor(z / Lz);
    int s = (int)floor(zw / dz);
    if (s >= S) s = S - 1;
    if (s < 0) s = 0;
    return s;
}

/* ---- transforms ------------------------------------------------------------------------ */

/* Brute-force DFT: out[k] = sum_j in[j] exp(sign 2 pi i j k / n), phase reduced mod n. */
void oracle_dft(const cplx *in, cplx *out, int n, int sign) {
    for (int k = 0; k < n; k++) {
        cplx acc = 0;
        for (int j = 0; j < n; j++) {
            long r = ((long)j * (long)k) % n;
            acc += in[j] * cexp(sign * 2.0 * M_PI * I * (double)r / (double)n);
        }
        out[k] = acc;
    }
}

/* O(N^4) 2D DFT of a row-major [ny][nx] array. */
void oracle_dft2_brute(const cplx *in, cplx *out, int ny, int nx, int sign) {
    for (int ky = 0; ky < ny; ky++)
        for (int kx = 0; kx < nx; kx++) {
            cplx acc = 0;
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    double ph = (double)(((long)x * kx) % nx) / nx + (double)(((long)y * ky) % ny) / ny;
                    acc += in[(size_t)y * nx + x] * cexp(sign * 2.0 * M_PI * I * ph);
                }
            out[(size_t)ky * nx + kx] = acc;
        }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

/* Mixed-radix decimation in time (Cooley-Tukey with the smallest prime factor p of n):
 * with m = n / p and y_r the length-m transform of the samples x[p j + r], r = 0..p-1,
 *   X[k + m q] = sum_r exp(sign 2 pi i r (k + m q) / n) y_r[k],   k < m, q < p.
 * A prime n reduces to the direct sum.  w[j * ws] = exp(sign 2 pi i j / n) is the twiddle
 * table of this length (a sub-transform of length m reads it with stride ws * p).  scratch
 * holds 2 n values: y in the first n, the sub-transforms' own scratch after it. */
static void fft_mixed(cplx *x, int n, const cplx *w, long ws, cplx *scratch) {
    if (n <= 1) return;
    const int p = smallest_factor(n), m = n / p;
    cplx *y = scratch;  /* y[r m + k] = y_r[k] */
    for (int r = 0; r < p; r++) {
        for (int j = 0; j < m; j++) y[(size_t)r * m + j] = x[(size_t)j * p + r];
        fft_mixed(y + (size_t)r * m, m, w, ws * p, scratch + n);
    }
    for (int q = 0; q < p; q++)
        for (int k = 0; k < m; k++) {
            const int kk = k + m * q;
            cplx acc = 0;
            long ph = 0;  /* r kk mod n, stepped by kk */
            for (int r = 0; r < p; r++) {
                acc += y[(size_t)r * m + k] * w[ph * ws];
                ph += kk;
                if (ph >= n) ph -= n;
            }
            x[kk] = acc;
        }
}

/* In-place unnormalised FFT; sign -1 forward, +1 inverse.  Powers of two take the radix-2
 * path below, every other n the mixed-radix one.  Twiddles from cos/sin of the exact angle. */
void oracle_fft(cplx *x, int n, int sign) {
    if (n <= 1) return;
    if (!is_pow2(n)) {
        cplx *w = malloc(sizeof(cplx) * (size_t)n);
        for (int j = 0; j < n; j++) {
            double a = 2.0 * M_PI * (double)j / (double)n;
            w[j] = cos(a) + sign * I * sin(a);
        }
        cplx *scratch = malloc(sizeof(cplx) * 2 * (size_t)n);
        fft_mixed(x, n, w, 1, scratch);
        free(scratch);
        free(w);
        return;
    }
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    cplx *w = malloc(sizeof(cplx) * (size_t)(n / 2));
    for (int j = 0; j < n / 2; j++) {
        double a = 2.0 * M_PI * (double)j / (double)n;
        w[j] = cos(a) + sign * I * sin(a);
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < half; j++) {
                cplx u = x[i + j], v = x[i + j + half] * w[j * step];
                x[i + j] = u + v;
                x[i + j + half] = u - v;
            }
    }
    free(w);
}

/* Unnormalised 2D FFT of a row-major [ny][nx] array: rows, then columns. */
void oracle_fft2(cplx *a, int ny, int nx, int sign) {
    for (int y = 0; y < ny; y++) oracle_fft(a + (size_t)y * nx, nx, sign);
    cplx *col = malloc(sizeof(cplx) * (size_t)ny);
    for (int x = 0; x < nx; x++) {
        for (int y = 0; y < ny; y++) col[y] = a[(size_t)y * nx + x];
        oracle_fft(col, ny, sign);
        for (int y = 0; y < ny; y++) a[(size_t)y * nx + x] = col[y];
    }
    free(col);
}

/* ---- potential ------------------------------------------------------------------------- */

/* Projected potential of slice s (V A) into V[ny][nx]:
 * V(k) = (2 pi a0 e / A) M(k) sum_{j in s} f_Zj(|k|) exp(-2 pi i k.r_j), then
 * v(r) = sum_k V(k) exp(2 pi i k.r) (unnormalised inverse DFT), real part kept.
 * exp(-2 pi i k.r) is evaluated as exp(-2 pi i kx x) exp(-2 pi i ky y).
 * Returns the number of atoms in the slice, or -1 for a species missing from the table. */
int oracle_potential_slice(const oracle_params *p, const float *pos, const int32_t *Z, int n_atoms,
                           int s, const int32_t *tabZ, const double *coef, int nZ, double *V) {
    const int nx = p->nx, ny = p->ny;
    const size_t nq = (size_t)nx * ny;
    cplx *acc = calloc(nq * (size_t)nZ, sizeof(cplx));
    cplx *ex = malloc(sizeof(cplx) * (size_t)nx), *ey = malloc(sizeof(cplx) * (size_t)ny);
    char *mask = malloc(nq);
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) mask[(size_t)iy * nx + ix] = (char)oracle_mask(p, iy, ix);
    int count = 0, bad = 0;
    for (int j = 0; j < n_atoms; j++) {
        double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
        if (oracle_slice_index(z, p->Lz, p->n_slices) != s) continue;
        int zi = -1;
        for (int i = 0; i < nZ; i++) if (tabZ[i] == Z[j]) zi = i;
        if (zi < 0) { bad = 1; continue; }
        count++;
        for (int ix = 0; ix < nx; ix++) ex[ix] = cexp(-2.0 * M_PI * I * oracle_kfreq(ix, nx, p->Lx) * x);
        for (int iy = 0; iy < ny; iy++) ey[iy] = cexp(-2.0 * M_PI * I * oracle_kfreq(iy, ny, p->Ly) * y);
        cplx *a = acc + nq * (size_t)zi;
        for (int iy = 0; iy < ny; iy++)
            for (int ix = 0; ix < nx; ix++)
                if (mask[(size_t)iy * nx + ix]) a[(size_t)iy * nx + ix] += ex[ix] * ey[iy];
    }
    const double pre = oracle_kirkland_prefactor() / (p->Lx * p->Ly);
    cplx *Vk = calloc(nq, sizeof(cplx));
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            if (!mask[(size_t)iy * nx + ix]) continue;
            double kx = oracle_kfreq(ix, nx, p->Lx), ky = oracle_kfreq(iy, ny, p->Ly);
            double q = sqrt(kx * kx + ky * ky);
            cplx sum = 0;
            for (int i = 0; i < nZ; i++) sum += oracle_form_factor(coef + 12 * i, q) * acc[nq * (size_t)i + (size_t)iy * nx + ix];
            Vk[(size_t)iy * nx + ix] = pre * sum;
        }
    oracle_fft2(Vk, ny, nx, +1);
    for (size_t i = 0; i < nq; i++) V[i] = creal(Vk[i]);
    free(Vk); free(acc); free(ex); free(ey); free(mask);
    return bad ? -1 : count;
}

/* ---- transmission, probe, propagation ---------------------------------------------------- */

/* t = exp(i sigma V); with the transmission band limit t <- IDFT(M DFT(t)) / Nq. */
void oracle_transmission(const oracle_params *p, const double *V, cplx *t) {
    const size_t nq = (size_t)p->nx * p->ny;
    const double sig = oracle_sigma(p->voltage_ev) * p->sigma_scale;
    for (size_t i = 0; i < nq; i++) t[i] = cexp(I * sig * V[i]);
    if (p->bandlimit_transmission && p->bandlimit > 0.0) {
        oracle_fft2(t, p->ny, p->nx, -1);
        for (int iy = 0; iy < p->ny; iy++)
            for (int ix = 0; ix < p->nx; ix++) {
                size_t i = (size_t)iy * p->nx + ix;
                t[i] = oracle_mask(p, iy, ix) ? t[i] / (double)nq : 0.0;
            }
        oracle_fft2(t, p->ny, p->nx, +1);
    }
}

/* Real-space initial wave for a probe at (xp, yp) A.  alpha_mrad <= 0: plane wave. */
void oracle_probe(const oracle_params *p, double alpha_mrad, double xp, double yp, cplx *psi) {
    const int nx = p->nx, ny = p->ny;
    const size_t nq = (size_t)nx * ny;
    if (alpha_mrad <= 0.0) {
        for (size_t i = 0; i < nq; i++) psi[i] = 1.0 / sqrt((double)nq);
        return;
    }
    const double kmax = alpha_mrad * 1e-3 / oracle_wavelength(p->voltage_ev);
    double norm2 = 0.0;
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double kx = oracle_kfreq(ix, nx, p->Lx), ky = oracle_kfreq(iy, ny, p->Ly);
            int in = (kx * kx + ky * ky) <= kmax * kmax;
            psi[(size_t)iy * nx + ix] = in ? cexp(-2.0 * M_PI * I * kx * xp) * cexp(-2.0 * M_PI * I * ky * yp) : 0.0;
            norm2 += in;
        }
    for (size_t i = 0; i < nq; i++) psi[i] /= sqrt(norm2);       /* sum_k |psi(k)|^2 = 1 */
    oracle_fft2(psi, ny, nx, +1);                                  /* unitary inverse: */
    for (size_t i = 0; i < nq; i++) psi[i] /= sqrt((double)nq);
}

/* One slice: psi <- IDFT(P M DFT(t psi)) / Nq, P = exp(-i pi lambda dz |k|^2).
 * propagate = 0 keeps the mask but drops P (used for the last slice when final_propagator=0). */
static void slice_step(const oracle_params *p, const cplx *t, cplx *psi, int propagate) {
    const int nx = p->nx, ny = p->ny;
    const size_t nq = (size_t)nx * ny;
    const double lam = oracle_wavelength(p->voltage_ev), dz = p->Lz / (double)p->n_slices;
    for (size_t i = 0; i < nq; i++) psi[i] *= t[i];
    oracle_fft2(psi, ny, nx, -1);
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            size_t i = (size_t)iy * nx + ix;
            if (!oracle_mask(p, iy, ix)) { psi[i] = 0.0; continue; }
            double kx = oracle_kfreq(ix, nx, p->Lx), ky = oracle_kfreq(iy, ny, p->Ly);
            cplx P = propagate ? cexp(-I * M_PI * lam * dz * (kx * kx + ky * ky)) : 1.0;
            psi[i] *= P / (double)nq;
        }
    oracle_fft2(psi, ny, nx, +1);
}

/* Multislice of one frame for P probes: psi_k[P][ny][nx] = DFT(psi_exit) / sqrt(Nq).
 * V_out (optional, [S][ny][nx]) receives the slice potentials.  Returns 0, or -1 when an
 * atom's species is missing from the table. */
int oracle_multislice_frame(const oracle_params *p, const float *pos, const int32_t *Z, int n_atoms,
                            const int32_t *tabZ, const double *coef, int nZ, double alpha_mrad,
                            const double *probes_xy, int n_probes, cplx *psi_k, double *V_out) {
    const size_t nq = (size_t)p->nx * p->ny;
    const int S = p->n_slices;
    double *V = malloc(sizeof(double) * nq);
    cplx *t = malloc(sizeof(cplx) * nq * (size_t)S);
    int rc = 0;
    for (int s = 0; s < S; s++) {
        if (oracle_potential_slice(p, pos, Z, n_atoms, s, tabZ, coef, nZ, V) < 0) rc = -1;
        if (V_out) memcpy(V_out + nq * (size_t)s, V, sizeof(double) * nq);
        oracle_transmission(p, V, t + nq * (size_t)s);
    }
    for (int ip = 0; ip < n_probes; ip++) {
        cplx *psi = psi_k + nq * (size_t)ip;
        oracle_probe(p, alpha_mrad, probes_xy[2 * ip], probes_xy[2 * ip + 1], psi);
        for (int s = 0; s < S; s++)
            slice_step(p, t + nq * (size_t)s, psi, (s < S - 1) || p->final_propagator);
        oracle_fft2(psi, p->ny, p->nx, -1);
        for (size_t i = 0; i < nq; i++) psi[i] /= sqrt((double)nq);
    }
    free(V); free(t);
    return rc;
}

/* All frames: psi_k[P][F][ny][nx]; frames run in parallel (OpenMP).  Returns 0 or -1. */
int oracle_multislice(const oracle_params *p, const float *pos, int n_frames, const int32_t *Z, int n_atoms,
                      const int32_t *tabZ, const double *coef, int nZ, double alpha_mrad,
                      const double *probes_xy, int n_probes, cplx *psi_k) {
    const size_t nq = (size_t)p->nx * p->ny;
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int f = 0; f < n_frames; f++) {
        cplx *tmp = malloc(sizeof(cplx) * nq * (size_t)n_probes);
        int r = oracle_multislice_frame(p, pos + (size_t)f * n_atoms * 3, Z, n_atoms, tabZ, coef, nZ,
                                        alpha_mrad, probes_xy, n_probes, tmp, NULL);
        if (r < rc) rc = r;
        for (int ip = 0; ip < n_probes; ip++)
            memcpy(psi_k + ((size_t)ip * n_frames + f) * nq, tmp + (size_t)ip * nq, sizeof(cplx) * nq);
        free(tmp);
    }
    return rc;
}

/* ---- time transform ---------------------------------------------------------------------- */

/* S[p][m][q] = |sum_n (psi[p][n][q] - mean_n psi[p][n][q]) exp(-2 pi i m n / F)|^2.
 * subtract_mean = 0 skips the mean; direct = 1 uses the O(F^2) sum instead of the FFT. */
void oracle_spectrum(const cplx *psi, int P, int F, long nq, int subtract_mean, int direct, double *S) {
#pragma omp parallel
    {
        cplx *r = malloc(sizeof(cplx) * (size_t)F), *o = malloc(sizeof(cplx) * (size_t)F);
#pragma omp for schedule(static)
        for (long pq = 0; pq < (long)P * nq; pq++) {
            long p = pq / nq, q = pq % nq;
            const cplx *col = psi + (size_t)p * F * nq + q;
            cplx mean = 0;
            if (subtract_mean) {
                for (int n = 0; n < F; n++) mean += col[(size_t)n * nq];
                mean /= (double)F;
            }
            for (int n = 0; n < F; n++) r[n] = col[(size_t)n * nq] - mean;
            if (direct) {
                oracle_dft(r, o, F, -1);
            } else {
                memcpy(o, r, sizeof(cplx) * (size_t)F);
                oracle_fft(o, F, -1);
            }
            double *Sc = S + (size_t)p * F * nq + q;
            for (int m = 0; m < F; m++) {
                double a = creal(o[m]), b = cimag(o[m]);
                Sc[(size_t)m * nq] = a * a + b * b;
            }
        }
        free(r); free(o);
    }
}

/* Mean over frames, FP64: mean[p][q] = (1/F) sum_n psi[p][n][q]. */
void oracle_mean(const cplx *psi, int P, int F, long nq, cplx *mean) {
    for (long p = 0; p < P; p++)
        for (long q = 0; q < nq; q++) {
            cplx m = 0;
            for (int n = 0; n < F; n++) m += psi[((size_t)p * F + n) * nq + q];
            mean[p * nq + q] = m / (double)F;
        }
}

/* ---- TACAW accessors (Methods, "Data Structure Design": dispersion, spectral diffraction,
 * spectrum image) and trajectory averaging (Methods, "Molecular Dynamics"; Supplement,
 * "Sampling Considerations") ---------------------------------------------------------------- */

/* Bin of frequency f (THz) on an F-point axis with spacing dt (fs): round(f F dt), in FFT order. */
int oracle_freq_bin(double f_thz, int F, double dt_fs) {
    long m = lround(f_thz * (double)F * dt_fs * 1e-3);
    m %= F;
    if (m < 0) m += F;
    return (int)m;
}

/* map[p][q] = S[p][m][q] (+ S[p][-m][q] when fold), m the bin of f. */
void oracle_spectral_diffraction(const double *S, int P, int F, long nq, double dt_fs, double f_thz, int fold,
                                 double *map) {
    int m = oracle_freq_bin(f_thz, F, dt_fs), mn = (F - m) % F;
    for (long p = 0; p < P; p++)
        for (long q = 0; q < nq; q++) {
            double v = S[((size_t)p * F + m) * nq + q];
            if (fold && mn != m) v += S[((size_t)p * F + mn) * nq + q];
            map[p * nq + q] = v;
        }
}

/* S(k, w) along a path: bilinear interpolation of S[p][m][ny][nx] at (kx, ky) (1/A) on the
 * periodic reciprocal grid (spacing 1/Lx, 1/Ly).  out[p][m][i]. */
void oracle_dispersion(const double *S, int P, int F, int ny, int nx, double Lx, double Ly, const double *kx,
                       const double *ky, int npts, double *out) {
    for (int p = 0; p < P; p++)
        for (int m = 0; m < F; m++) {
            const double *plane = S + ((size_t)p * F + m) * (size_t)ny * nx;
            for (int i = 0; i < npts; i++) {
                double u = kx[i] * Lx, v = ky[i] * Ly;      /* fractional grid indices */
                double u0 = floor(u), v0 = floor(v), fu = u - u0, fv = v - v0;
                long iu = ((long)u0 % nx + nx) % nx, iv = ((long)v0 % ny + ny) % ny;
                long iu1 = (iu + 1) % nx, iv1 = (iv + 1) % ny;
                double s00 = plane[iv * nx + iu], s01 = plane[iv * nx + iu1];
                double s10 = plane[iv1 * nx + iu], s11 = plane[iv1 * nx + iu1];
                out[((size_t)p * F + m) * npts + i] =
                    (1 - fv) * ((1 - fu) * s00 + fu * s01) + fv * ((1 - fu) * s10 + fu * s11);
            }
        }
}

/* Convergent probe with aberrations (Discussion, "Beyond Vibrational Spectroscopy": the
 * standard aberration function with defocus, astigmatism, coma and spherical aberration):
 * psi0(k) = A(k) exp(-i chi(k)) exp(-2 pi i k.r_p) / norm, with, at theta = lambda k,
 * chi = (2 pi / lambda) (df theta^2 / 2 + a1 theta^2 cos 2(phi - phi_a) / 2
 *                        + b2 theta^3 cos(phi - phi_b) / 3 + Cs theta^4 / 4)
 * (df, a1, b2 in A, Cs in mm), then a unitary inverse transform.  With chi = 0 this is
 * oracle_probe. */
void oracle_probe_aberrated(const oracle_params *p, double alpha_mrad, double xp, double yp, double df_A,
                            double cs_mm, double a1_A, double phi_a, double b2_A, double phi_b, cplx *psi) {
    const int nx = p->nx, ny = p->ny;
    const size_t nq = (size_t)nx * ny;
    const double lam = oracle_wavelength(p->voltage_ev);
    const double kmax = alpha_mrad * 1e-3 / lam, cs = cs_mm * 1e7;
    double norm2 = 0.0;
    for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
            double kx = oracle_kfreq(ix, nx, p->Lx), ky = oracle_kfreq(iy, ny, p->Ly);
            double k2 = kx * kx + ky * ky;
            int in = k2 <= kmax * kmax;
            double theta = lam * sqrt(k2), phi = atan2(ky, kx);
            double chi = (2.0 * M_PI / lam) * (0.5 * df_A * theta * theta +
                                               0.5 * a1_A * theta * theta * cos(2.0 * (phi - phi_a)) +
                                               b2_A * theta * theta * theta * cos(phi - phi_b) / 3.0 +
                                               0.25 * cs * theta * theta * theta * theta);
            psi[(size_t)iy * nx + ix] = in ? cexp(-I * chi) * cexp(-2.0 * M_PI * I * kx * xp) *
                                                 cexp(-2.0 * M_PI * I * ky * yp)
                                           : 0.0;
            norm2 += in;
        }
    for (size_t i = 0; i < nq; i++) psi[i] /= sqrt(norm2);
    oracle_fft2(psi, ny, nx, +1);
    for (size_t i = 0; i < nq; i++) psi[i] /= sqrt((double)nq);
}

/* Multislice of one frame from given real-space initial waves psi0[P][ny][nx] (any probe:
 * aberrated, vortex, ...): psi_k[P][ny][nx] = DFT(psi_exit) / sqrt(Nq).  Returns 0 or -1. */
int oracle_multislice_frame_init(const oracle_params *p, const float *pos, const int32_t *Z, int n_atoms,
                                 const int32_t *tabZ, const double *coef, int nZ, const cplx *psi0, int n_probes,
                                 cplx *psi_k) {
    const size_t nq = (size_t)p->nx * p->ny;
    const int S = p->n_slices;
    double *V = malloc(sizeof(double) * nq);
    cplx *t = malloc(sizeof(cplx) * nq * (size_t)S);
    int rc = 0;
    for (int s = 0; s < S; s++) {
        if (oracle_potential_slice(p, pos, Z, n_atoms, s, tabZ, coef, nZ, V) < 0) rc = -1;
        oracle_transmission(p, V, t + nq * (size_t)s);
    }
    for (int ip = 0; ip < n_probes; ip++) {
        cplx *psi = psi_k + nq * (size_t)ip;
        memcpy(psi, psi0 + nq * (size_t)ip, sizeof(cplx) * nq);
        for (int s = 0; s < S; s++)
            slice_step(p, t + nq * (size_t)s, psi, (s < S - 1) || p->final_propagator);
        oracle_fft2(psi, p->ny, p->nx, -1);
        for (size_t i = 0; i < nq; i++) psi[i] /= sqrt((double)nq);
    }
    free(V); free(t);
    return rc;
}

/*
 * FP64 CPU oracle for the SOE-Ewald2D long-range sums (test infrastructure).
 *
 * ORACLE: this file is test infrastructure. Only tests/, the smoke check and
 * the CPU baseline of the benchmark call it. It shares no code with the CUDA
 * library and is deliberately plain: one complex recursion per (k, beta), in
 * the order and notation of the paper, with no blocking or reordering.
 *
 * What it computes (Gan, Gao, Liang, Xu, "Fast algorithm for quasi-2D Coulomb
 * systems"):
 *
 *   k != 0 (Section 3.2, Eq. 3.21 and Eqs. 3.27-3.30; forces Appendix E):
 *     For a mode k and a parameter beta with Re(beta) > 0, with particles
 *     sorted so that z_1 <= ... <= z_N and u_j = q_j e^{-i k.rho_j}:
 *       A_1 = 0,  A_i = A_{i-1} e^{-beta (z_{i-1} - z_{i-2})} + u_{i-1},
 *       F_i = e^{-beta (z_i - z_{i-1})} A_i = sum_{j<i} u_j e^{-beta(z_i-z_j)},
 *     and the mirrored backward recursion for B_i = sum_{j>i} u_j
 *     e^{-beta(z_j-z_i)} (Appendix E needs both the j<i and the j>i sums).
 *     The SOE pair kernel of Eq. 3.21 is
 *       (1/k)(xi+_M + xi-_M)(k,z) = C_k sum_l w_l (2 a_l e^{-kz} - 2k e^{-a_l z})
 *                                   / (a_l^2 - k^2),   a_l = alpha s_l,
 *     so beta runs over {k, a_1..a_M} with coefficients
 *       c_k = sum_l 2 a_l w_l/(a_l^2-k^2),  c_l = -2 k w_l/(a_l^2-k^2).
 *     With T_i = sum_beta c_beta (F_i + B_i) and Tz_i = sum_beta c_beta beta
 *     (F_i - B_i), each mode adds (gam_k = its prefactor, see below)
 *       phi_i  += gam_k Re[e^{i k.rho_i} T_i]
 *       F_rho  += gam_k q_i kvec Im[e^{i k.rho_i} T_i]
 *       F_z    += gam_k q_i Re[e^{i k.rho_i} Tz_i]
 *     where F = -grad E and E = 1/2 sum_i q_i phi_i (the signs follow from
 *     differentiating the pair form; the printed leading minus of the
 *     Appendix E gradient is not used).
 *
 *   k = 0 (Eqs. 3.24-3.26, derivative Eq. E.6): the SOE form of
 *     g0(z) = z erf(alpha z) + e^{-alpha^2 z^2}/(alpha sqrt(pi)) is
 *       g0_SOE(z) = sum_l (w_l/sqrt(pi)) [2z/s_l + (1/alpha - 2z/s_l) e^{-a_l z}],
 *     and
 *       phi0_i = -(2 pi/A) sum_{j != i} q_j g0_SOE(|z_i - z_j|)
 *       F0_z,i = (2 pi/A) q_i sum_{j != i} q_j g0_SOE'(|z_ij|) sgn(z_i - z_j).
 *     The |z| parts use sorted prefix sums of q and q z; the exponential parts
 *     use the same A_i recursion with inputs q_j and q_j z_j.
 *
 *   k-derivative of the k != 0 pair sums (the lateral virial, oracle/virial.py):
 *     R_k = sum_{i != j} q_i q_j cos(k.rho_ij) d/dk G_SOE(k, |z_ij|),
 *     G_SOE(k, z) = C_k sum_beta c_beta e^{-beta z}.
 *     Only C_k, the coefficients c_beta and the node beta = k depend on k
 *     (a_l = alpha s_l does not), so
 *       dG_SOE/dk = sum_beta (C_k c_beta)' e^{-beta z} - C_k c_k z e^{-k z},
 *     C_k' = C_k (-k/(2 alpha^2) - 1/k),
 *     c_k' = sum_l 4 k a_l w_l/(a_l^2-k^2)^2,
 *     c_l' = -2 w_l (a_l^2+k^2)/(a_l^2-k^2)^2.
 *     The pair sums are sum_i conj(u_i) (F_i + B_i) (their sin part cancels
 *     between (i,j) and (j,i)); the z-weighted sum for beta = k is
 *     sum_{j<i} u_j (z_i - z_j) e^{-k(z_i-z_j)} = z_i F_i(u) - F_i(u z) and
 *     its mirror B_i(u z) - z_i B_i(u).
 *
 * The diagonal (j = i) constants, the self term and the energy are added by
 * the Python wrapper.
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

struct key { double z; int64_t i; };

static int cmp_key(const void* a, const void* b) {
    const struct key* p = (const struct key*)a;
    const struct key* q = (const struct key*)b;
    if (p->z < q->z) return -1;
    if (p->z > q->z) return 1;
    return (p->i < q->i) ? -1 : (p->i > q->i);
}

/* Sorted order by z, ties broken by the original index (a stable order). */
static int64_t* sort_by_z(int64_t N, const double* z) {
    struct key* k = (struct key*)malloc(sizeof(struct key) * (size_t)(N > 0 ? N : 1));
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) { k[i].z = z[i]; k[i].i = i; }
    qsort(k, (size_t)N, sizeof(struct key), cmp_key);
    for (int64_t i = 0; i < N; ++i) ord[i] = k[i].i;
    free(k);
    return ord;
}

/* Forward sums F_i = sum_{j<i} u_j e^{-beta (z_i - z_j)} by the A_i recursion.
 * dec[i] = e^{-beta (z_i - z_{i-1})} for i >= 1 (dec[0] unused). */
static void forward_sum(int64_t N, const cplx* u, const cplx* dec, cplx* F) {
    cplx A = 0.0;                       /* A_1 = 0 */
    if (N > 0) F[0] = 0.0;
    for (int64_t i = 1; i < N; ++i) {
        if (i >= 2) A = A * dec[i - 1] + u[i - 1];
        else        A = u[0];           /* A_2 = u_1 */
        F[i] = dec[i] * A;
    }
}

/* Backward sums B_i = sum_{j>i} u_j e^{-beta (z_j - z_i)}, mirrored. */
static void backward_sum(int64_t N, const cplx* u, const cplx* dec, cplx* B) {
    cplx A = 0.0;
    if (N > 0) B[N - 1] = 0.0;
    for (int64_t i = N - 2; i >= 0; --i) {
        if (i <= N - 3) A = A * dec[i + 2] + u[i + 1];
        else            A = u[N - 1];
        B[i] = dec[i + 1] * A;
    }
}

/*
 * k != 0 part. Inputs in the caller's order; outputs in the caller's order
 * (phi, fx, fy, fz are overwritten). Modes: K vectors (kx, ky) with prefactor
 * gam[k] (the caller folds pi/(Lx Ly), C_k and the sampling weight into it).
 * SOE: M complex (s_l, w_l) given as separate real/imaginary arrays.
 */
void oracle_kspace_soe(int64_t N, const double* x, const double* y,
                       const double* z, const double* q, int64_t K,
                       const double* kx, const double* ky, const double* gam,
                       double alpha, int M, const double* s_re,
                       const double* s_im, const double* w_re,
                       const double* w_im, double* phi, double* fx,
                       double* fy, double* fz) {
    int64_t* ord = sort_by_z(N, z);
    double *xs = malloc(sizeof(double) * N), *ys = malloc(sizeof(double) * N);
    double *zs = malloc(sizeof(double) * N), *qs = malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) {
        xs[i] = x[ord[i]]; ys[i] = y[ord[i]]; zs[i] = z[ord[i]]; qs[i] = q[ord[i]];
    }
    cplx* a = malloc(sizeof(cplx) * (M > 0 ? M : 1));
    cplx* wl = malloc(sizeof(cplx) * (M > 0 ? M : 1));
    for (int l = 0; l < M; ++l) {
        a[l] = alpha * (s_re[l] + I * s_im[l]);
        wl[l] = w_re[l] + I * w_im[l];
    }
    /* k-independent decays e^{-a_l (z_i - z_{i-1})}. */
    cplx* decl = malloc(sizeof(cplx) * (size_t)(M > 0 ? M : 1) * (size_t)(N > 0 ? N : 1));
    for (int l = 0; l < M; ++l) {
        decl[(size_t)l * N] = 1.0;
        for (int64_t i = 1; i < N; ++i)
            decl[(size_t)l * N + i] = cexp(-a[l] * (zs[i] - zs[i - 1]));
    }
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double* acc = calloc((size_t)nth * 4 * (size_t)N, sizeof(double));

#pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* aphi = acc + (size_t)tid * 4 * N;
        double* afx = aphi + N;
        double* afy = afx + N;
        double* afz = afy + N;
        cplx* u = malloc(sizeof(cplx) * N);
        cplx* deck = malloc(sizeof(cplx) * N);
        cplx* F = malloc(sizeof(cplx) * N);
        cplx* B = malloc(sizeof(cplx) * N);
        cplx* T = malloc(sizeof(cplx) * N);
        cplx* Tz = malloc(sizeof(cplx) * N);
#pragma omp for schedule(static)
        for (int64_t m = 0; m < K; ++m) {
            double k = sqrt(kx[m] * kx[m] + ky[m] * ky[m]);
            for (int64_t i = 0; i < N; ++i) {
                u[i] = qs[i] * cexp(-I * (kx[m] * xs[i] + ky[m] * ys[i]));
                T[i] = 0.0;
                Tz[i] = 0.0;
            }
            /* beta = k */
            cplx ck = 0.0;
            for (int l = 0; l < M; ++l)
                ck += 2.0 * a[l] * wl[l] / (a[l] * a[l] - k * k);
            deck[0] = 1.0;
            for (int64_t i = 1; i < N; ++i) deck[i] = exp(-k * (zs[i] - zs[i - 1]));
            forward_sum(N, u, deck, F);
            backward_sum(N, u, deck, B);
            for (int64_t i = 0; i < N; ++i) {
                T[i] += ck * (F[i] + B[i]);
                Tz[i] += ck * k * (F[i] - B[i]);
            }
            /* beta = a_l */
            for (int l = 0; l < M; ++l) {
                cplx cl = -2.0 * k * wl[l] / (a[l] * a[l] - k * k);
                forward_sum(N, u, decl + (size_t)l * N, F);
                backward_sum(N, u, decl + (size_t)l * N, B);
                for (int64_t i = 0; i < N; ++i) {
                    T[i] += cl * (F[i] + B[i]);
                    Tz[i] += cl * a[l] * (F[i] - B[i]);
                }
            }
            for (int64_t i = 0; i < N; ++i) {
                cplx ph = cexp(I * (kx[m] * xs[i] + ky[m] * ys[i]));
                cplx Z = ph * T[i];
                cplx Zz = ph * Tz[i];
                aphi[i] += gam[m] * creal(Z);
                afx[i] += gam[m] * qs[i] * kx[m] * cimag(Z);
                afy[i] += gam[m] * qs[i] * ky[m] * cimag(Z);
                afz[i] += gam[m] * qs[i] * creal(Zz);
            }
        }
        free(u); free(deck); free(F); free(B); free(T); free(Tz);
    }
    for (int64_t i = 0; i < N; ++i) {
        double p = 0, gx = 0, gy = 0, gz = 0;
        for (int t = 0; t < nth; ++t) {
            const double* base = acc + (size_t)t * 4 * N;
            p += base[i]; gx += base[N + i]; gy += base[2 * N + i]; gz += base[3 * N + i];
        }
        int64_t o = ord[i];
        phi[o] = p; fx[o] = gx; fy[o] = gy; fz[o] = gz;
    }
    free(acc); free(decl); free(a); free(wl);
    free(xs); free(ys); free(zs); free(qs); free(ord);
}

/*
 * k = 0 part (pair terms only): phi0[i] = -(2 pi/A) sum_{j!=i} q_j g0_SOE(|z_ij|)
 * and fz0[i] = (2 pi/A) q_i sum_{j!=i} q_j g0_SOE'(|z_ij|) sgn(z_i - z_j).
 */
void oracle_kzero_soe(int64_t N, const double* z, const double* q, double area,
                      double alpha, int M, const double* s_re,
                      const double* s_im, const double* w_re,
                      const double* w_im, double* phi0, double* fz0) {
    const double pi = 3.14159265358979323846;
    int64_t* ord = sort_by_z(N, z);
    double *zs = malloc(sizeof(double) * N), *qs = malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) { zs[i] = z[ord[i]]; qs[i] = q[ord[i]]; }
    /* exclusive prefix / suffix sums of q and q z (FP64) */
    double *Qlt = malloc(sizeof(double) * N), *Qgt = malloc(sizeof(double) * N);
    double *Plt = malloc(sizeof(double) * N), *Pgt = malloc(sizeof(double) * N);
    double s0 = 0, s1 = 0;
    for (int64_t i = 0; i < N; ++i) { Qlt[i] = s0; Plt[i] = s1; s0 += qs[i]; s1 += qs[i] * zs[i]; }
    s0 = 0; s1 = 0;
    for (int64_t i = N - 1; i >= 0; --i) { Qgt[i] = s0; Pgt[i] = s1; s0 += qs[i]; s1 += qs[i] * zs[i]; }

    cplx* pot = calloc((size_t)N, sizeof(cplx));   /* sum_j q_j g0(|z_ij|)       */
    cplx* der = calloc((size_t)N, sizeof(cplx));   /* sum_j q_j g0'(|z_ij|) sgn  */
    cplx *uq = malloc(sizeof(cplx) * N), *uqz = malloc(sizeof(cplx) * N);
    cplx *dec = malloc(sizeof(cplx) * N);
    cplx *Sf = malloc(sizeof(cplx) * N), *Sb = malloc(sizeof(cplx) * N);
    cplx *Zf = malloc(sizeof(cplx) * N), *Zb = malloc(sizeof(cplx) * N);
    for (int64_t i = 0; i < N; ++i) { uq[i] = qs[i]; uqz[i] = qs[i] * zs[i]; }
    for (int l = 0; l < M; ++l) {
        cplx sl = s_re[l] + I * s_im[l];
        cplx wv = w_re[l] + I * w_im[l];
        cplx al = alpha * sl;
        dec[0] = 1.0;
        for (int64_t i = 1; i < N; ++i) dec[i] = cexp(-al * (zs[i] - zs[i - 1]));
        forward_sum(N, uq, dec, Sf);  backward_sum(N, uq, dec, Sb);
        forward_sum(N, uqz, dec, Zf); backward_sum(N, uqz, dec, Zb);
        cplx c = wv / sqrt(pi);
        for (int64_t i = 0; i < N; ++i) {
            double zi = zs[i];
            double lin = zi * Qlt[i] - Plt[i] + Pgt[i] - zi * Qgt[i];  /* sum_j q_j |z_ij| */
            cplx Hf = zi * Sf[i] - Zf[i];        /* sum_{j<i} q_j (z_i-z_j) e^{-a(z_i-z_j)} */
            cplx Hb = Zb[i] - zi * Sb[i];        /* sum_{j>i} q_j (z_j-z_i) e^{-a(z_j-z_i)} */
            pot[i] += c * (2.0 / sl * lin + (1.0 / alpha) * (Sf[i] + Sb[i]) - 2.0 / sl * (Hf + Hb));
            der[i] += c * (2.0 / sl * (Qlt[i] - Qgt[i]) - (2.0 / sl + sl) * (Sf[i] - Sb[i])
                           + 2.0 * alpha * (Hf - Hb));
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = ord[i];
        phi0[o] = -(2.0 * pi / area) * creal(pot[i]);
        fz0[o] = (2.0 * pi / area) * qs[i] * creal(der[i]);
    }
    free(pot); free(der); free(uq); free(uqz); free(dec);
    free(Sf); free(Sb); free(Zf); free(Zb);
    free(Qlt); free(Qgt); free(Plt); free(Pgt); free(zs); free(qs); free(ord);
}

/*
 * R[m] = sum_{i != j} q_i q_j cos(k.rho_ij) dG_SOE/dk(k, |z_ij|) for each
 * mode (kx[m], ky[m]); see the header comment. Inputs in any order.
 */
void oracle_kspace_soe_dk(int64_t N, const double* x, const double* y,
                          const double* z, const double* q, int64_t K,
                          const double* kx, const double* ky, double alpha,
                          int M, const double* s_re, const double* s_im,
                          const double* w_re, const double* w_im, double* R) {
    const double pi = 3.14159265358979323846;
    int64_t* ord = sort_by_z(N, z);
    double *xs = malloc(sizeof(double) * N), *ys = malloc(sizeof(double) * N);
    double *zs = malloc(sizeof(double) * N), *qs = malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) {
        xs[i] = x[ord[i]]; ys[i] = y[ord[i]]; zs[i] = z[ord[i]]; qs[i] = q[ord[i]];
    }
    cplx* a = malloc(sizeof(cplx) * (M > 0 ? M : 1));
    cplx* wl = malloc(sizeof(cplx) * (M > 0 ? M : 1));
    for (int l = 0; l < M; ++l) {
        a[l] = alpha * (s_re[l] + I * s_im[l]);
        wl[l] = w_re[l] + I * w_im[l];
    }
    cplx* decl = malloc(sizeof(cplx) * (size_t)(M > 0 ? M : 1) * (size_t)(N > 0 ? N : 1));
    for (int l = 0; l < M; ++l) {
        decl[(size_t)l * N] = 1.0;
        for (int64_t i = 1; i < N; ++i)
            decl[(size_t)l * N + i] = cexp(-a[l] * (zs[i] - zs[i - 1]));
    }
#pragma omp parallel
    {
        cplx* u = malloc(sizeof(cplx) * N);
        cplx* uz = malloc(sizeof(cplx) * N);
        cplx* deck = malloc(sizeof(cplx) * N);
        cplx *F = malloc(sizeof(cplx) * N), *B = malloc(sizeof(cplx) * N);
        cplx *Fz = malloc(sizeof(cplx) * N), *Bz = malloc(sizeof(cplx) * N);
#pragma omp for schedule(static)
        for (int64_t m = 0; m < K; ++m) {
            double k = sqrt(kx[m] * kx[m] + ky[m] * ky[m]);
            double Ck = 2.0 * alpha * exp(-k * k / (4.0 * alpha * alpha)) / (sqrt(pi) * k);
            double g = -k / (2.0 * alpha * alpha) - 1.0 / k;     /* C_k'/C_k */
            for (int64_t i = 0; i < N; ++i) {
                u[i] = qs[i] * cexp(-I * (kx[m] * xs[i] + ky[m] * ys[i]));
                uz[i] = u[i] * zs[i];
            }
            cplx ck = 0.0, dck = 0.0;
            for (int l = 0; l < M; ++l) {
                cplx den = a[l] * a[l] - k * k;
                ck += 2.0 * a[l] * wl[l] / den;
                dck += 4.0 * k * a[l] * wl[l] / (den * den);
            }
            /* beta = k: plain and z-weighted sums */
            deck[0] = 1.0;
            for (int64_t i = 1; i < N; ++i) deck[i] = exp(-k * (zs[i] - zs[i - 1]));
            forward_sum(N, u, deck, F);
            backward_sum(N, u, deck, B);
            forward_sum(N, uz, deck, Fz);
            backward_sum(N, uz, deck, Bz);
            cplx Pk = 0.0, Pz = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                cplx cu = conj(u[i]);
                Pk += cu * (F[i] + B[i]);
                Pz += cu * ((zs[i] * F[i] - Fz[i]) + (Bz[i] - zs[i] * B[i]));
            }
            cplx acc = Ck * (ck * g + dck) * Pk - Ck * ck * Pz;
            /* beta = a_l */
            for (int l = 0; l < M; ++l) {
                cplx den = a[l] * a[l] - k * k;
                cplx cl = -2.0 * k * wl[l] / den;
                cplx dcl = -2.0 * wl[l] * (a[l] * a[l] + k * k) / (den * den);
                forward_sum(N, u, decl + (size_t)l * N, F);
                backward_sum(N, u, decl + (size_t)l * N, B);
                cplx Pl = 0.0;
                for (int64_t i = 0; i < N; ++i) Pl += conj(u[i]) * (F[i] + B[i]);
                acc += Ck * (cl * g + dcl) * Pl;
            }
            R[m] = creal(acc);
        }
        free(u); free(uz); free(deck); free(F); free(B); free(Fz); free(Bz);
    }
    free(decl); free(a); free(wl);
    free(xs); free(ys); free(zs); free(qs); free(ord);
}

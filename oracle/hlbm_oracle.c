/*
 * FP64 reference solver for one time step of the high-order BGK lattice
 * Boltzmann method with Hermite body sources (Li et al., "Constructing the
 * body source for high-order lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the GPU path is checked
 * against.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA library: lattice velocities,
 * weights and c0^2 arrive from oracle/lattice.py through or_lattice.
 *
 * What it computes, in the paper's order and notation (lattice units,
 * dx = dt = 1, integer velocities c_i, xi_i = c_i / c0, cs2 = c0^2):
 *
 *   state: f[i][n] = f^_i(x_n, t), the shifted populations after streaming
 *          (Eq. 4.3).
 *   1. macroscopic fields at time t at EVERY node first (no time lag):
 *        rho   = sum_i f^_i                                   (Eq. 4.5)
 *        psi   = sqrt(2 (p_EOS(rho) - rho cs2) / (G cs2)), G = -1  (Eq. 3.8,
 *                with the lattice-unit normalisation of the sound speed)
 *        F^SC  = -G psi(x) sum_i w_i psi(x + c_i) c_i          (Eq. 3.8)
 *        F     = rho g(x) + F^SC     (force density; g an acceleration)
 *        u     = (sum_i c_i f^_i + F / 2) / rho               (Eq. 4.5)
 *        theta = (sum_i |c_i|^2 f^_i - rho |u|^2 + G2 / 2) / (rho D cs2),
 *                G2 = sum_i |c_i|^2 S_i = 2 u.F + sum_i |c_i|^2 P_i (Eq. 4.5)
 *        (theta-bar = theta - 1 enters f^eq and F_i only in thermal mode;
 *         the multiphase runs keep theta == 1, Sec. 5.4)
 *   2. grad theta by second-order central differences (Sec. 3.2).
 *   3. per node and velocity, the literal Table 2 polynomials:
 *        f^eq_i (Eq. 2.2 scaled), F_i (Eq. 3.3 scaled), H_i (Eq. 3.7
 *        scaled), P_i (Eq. 3.12 scaled); S_i = F_i + H_i + P_i.
 *   4. collision, Eq. 4.4:
 *        f*_i = f^_i - (f^_i - f^eq_i) / tau^ + (1 - 1 / (2 tau^)) S_i
 *   5. streaming: f^_i(x + c_i, t + 1) = f*_i(x), periodic in every axis.
 *
 * Readings of garbled or silent passages:
 *   - Table 2, F_i: the last term is -(c.u)(u.F)/c0^4 as in Eq. 3.3; the
 *     printed -(c.u)(c.F)/c0^4 would cancel the second term.
 *   - Table 2, H_i: factor (1 - 1/Pr) as in Eq. 3.7; the printed
 *     (1 - 1/(c0^2 Pr)) contradicts Eq. 3.6.
 *   - Eq. 4.5: u = (F^_1 + G_1 / 2) / rho (G_1 = F is a force density).
 *   - P_i: tau is the continuous relaxation time tau^ - 1/2 (Eq. 4.3).
 *   - D3Q39 (not in the paper): f^eq truncated after the third order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 64

typedef struct {
    int D, Q;
    int c[OR_MAXQ][3];
    double w[OR_MAXQ];
    double cs2;
} or_lattice;

typedef struct {
    int nx, ny, nz;
    double tau_hat;
    int feq_order;      /* 4: all of Eq. 2.2; 3: its first two lines */
    int thermal;        /* 1: theta-bar from the moments; 0: theta == 1 */
    int use_force;      /* body force F = rho g */
    double g_uniform[3];
    int use_H;          /* thermal diffusion source, Eq. 3.7 */
    double Pr;
    int use_SC;         /* pseudopotential force, Eq. 3.8 */
    int use_P;          /* pressure tensor source, Eq. 3.12 */
    int eos;            /* 0: van der Waals, 1: Carnahan-Starling (Eq. 5.9) */
    double eos_a, eos_b, eos_T;
    double k;           /* free parameter of Eq. 3.12 */
} or_params;

#define G_SC (-1.0)

static inline long wrapi(long x, long n) { long r = x % n; return r < 0 ? r + n : r; }

static inline long nbr(const or_params* P, long n, const int* c) {
    long nx = P->nx, ny = P->ny, nz = P->nz;
    long x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    x = wrapi(x + c[0], nx);
    y = wrapi(y + c[1], ny);
    z = wrapi(z + c[2], nz);
    return x + nx * (y + ny * z);
}

/* Equations of state in lattice units. */
double or_peos(const or_params* P, double rho) {
    double a = P->eos_a, b = P->eos_b, T = P->eos_T;
    if (P->eos == 0) {                       /* van der Waals */
        return rho * T / (1.0 - b * rho) - a * rho * rho;
    } else {                                 /* Carnahan-Starling, Eq. 5.9 with R = 1 */
        double e = b * rho / 4.0;
        double num = 1.0 + e + e * e - e * e * e;
        double den = (1.0 - e) * (1.0 - e) * (1.0 - e);
        return rho * T * num / den - a * rho * rho;
    }
}

/* Pseudopotential of Eq. 3.8 with theta == 1, in lattice units. */
double or_psi(const or_params* P, double cs2, double rho) {
    double s = 2.0 * (or_peos(P, rho) - rho * cs2) / (G_SC * cs2);
    return sqrt(s > 0.0 ? s : 0.0);
}

/* Table 2, first row: f^eq_i(rho, u, theta) for all i (Eq. 2.2 scaled by xi = c / c0). */
void or_feq(const or_lattice* L, int order, double rho, const double* u, double theta, double* feq) {
    const int D = L->D;
    const double s = L->cs2, tb = theta - 1.0;
    double uu = 0.0;
    for (int a = 0; a < D; ++a) uu += u[a] * u[a];
    for (int i = 0; i < L->Q; ++i) {
        double cu = 0.0, cc = 0.0;
        for (int a = 0; a < D; ++a) { cu += L->c[i][a] * u[a]; cc += (double)L->c[i][a] * L->c[i][a]; }
        double t = 1.0
                 + cu / s
                 + cu * cu / (2.0 * s * s)
                 - uu / (2.0 * s)
                 + tb * (cc - s * D) / (2.0 * s);
        t += cu * cu * cu / (6.0 * s * s * s)
           - cu * uu / (2.0 * s * s)
           + cu * tb * (cc - s * (D + 2)) / (2.0 * s * s);
        if (order >= 4) {
            t += cu * cu * cu * cu / (24.0 * s * s * s * s)
               - cu * cu * uu / (4.0 * s * s * s)
               + uu * uu / (8.0 * s * s);
            t += tb * (cu * cu * (cc - s * (D + 4)) + s * uu * (s * (D + 2) - cc)) / (4.0 * s * s * s);
            t += tb * tb * (cc * cc - 2.0 * s * (D + 2) * cc + s * s * D * (D + 2)) / (8.0 * s * s);
        }
        feq[i] = L->w[i] * rho * t;
    }
}

/* Source terms of Table 2 at one node.  Any output pointer may be NULL.
 *   SF: body force F_i (Eq. 3.3), F the total force density, theta-bar as given
 *   SH: thermal diffusion H_i (Eq. 3.7), needs rho, theta and grad theta
 *   SP: pressure tensor P_i (Eq. 3.12), needs |F^SC|^2 and psi
 */
void or_sources(const or_lattice* L, const or_params* P, double rho, const double* u, double theta,
                const double* F, const double* gradT, const double* Fsc, double psi,
                double* SF, double* SH, double* SP) {
    const int D = L->D;
    const double s = L->cs2;
    const double tb = P->thermal ? theta - 1.0 : 0.0;
    double uu = 0.0, uF = 0.0, Fsc2 = 0.0;
    for (int a = 0; a < D; ++a) { uu += u[a] * u[a]; uF += u[a] * F[a]; }
    if (Fsc) for (int a = 0; a < D; ++a) Fsc2 += Fsc[a] * Fsc[a];
    const double tau = P->tau_hat - 0.5;
    for (int i = 0; i < L->Q; ++i) {
        double cu = 0.0, cF = 0.0, cc = 0.0, cg = 0.0;
        for (int a = 0; a < D; ++a) {
            cu += L->c[i][a] * u[a];
            cF += L->c[i][a] * F[a];
            cc += (double)L->c[i][a] * L->c[i][a];
            if (gradT) cg += L->c[i][a] * gradT[a];
        }
        if (SF) {
            SF[i] = L->w[i] * (cF / s + cu * cF / (s * s) - uF / s
                    + cF * (cu * cu + tb * s * cc - s * uu - tb * s * s * (D + 2)) / (2.0 * s * s * s)
                    - cu * uF / (s * s));
        }
        if (SH) {
            SH[i] = L->w[i] * rho * theta * (1.0 - 1.0 / P->Pr) * (cc - s * (D + 2)) * cg / (2.0 * s);
        }
        if (SP) {
            double q = (psi > 0.0) ? Fsc2 / (psi * psi * G_SC) : 0.0;
            SP[i] = -L->w[i] * P->k / (2.0 * D * tau) * q * (cc - s * D);
        }
    }
}

/* Step 1: macroscopic fields at every node (two passes: rho/psi, then the rest). */
void or_macros(const or_lattice* L, const or_params* P, const double* f, const double* gfield,
               double* rho, double* u, double* theta, double* F, double* psi, double* Fsc) {
    const long N = (long)P->nx * P->ny * P->nz;
    const int D = L->D, Q = L->Q;
    const double s = L->cs2;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += f[(long)i * N + n];
        rho[n] = r;
        psi[n] = P->use_SC ? or_psi(P, s, r) : 0.0;
    }
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double fs[3] = {0.0, 0.0, 0.0};
        if (P->use_SC) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < Q; ++i) {
                double p = psi[nbr(P, n, L->c[i])];
                for (int a = 0; a < D; ++a) acc[a] += L->w[i] * p * L->c[i][a];
            }
            for (int a = 0; a < D; ++a) fs[a] = -G_SC * psi[n] * acc[a];
        }
        double Fn[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < D; ++a) {
            double g = 0.0;
            if (P->use_force) g = gfield ? gfield[(long)a * N + n] : P->g_uniform[a];
            Fn[a] = rho[n] * g + fs[a];
        }
        double j[3] = {0.0, 0.0, 0.0}, e = 0.0;
        for (int i = 0; i < Q; ++i) {
            double fi = f[(long)i * N + n];
            double cc = 0.0;
            for (int a = 0; a < D; ++a) { j[a] += L->c[i][a] * fi; cc += (double)L->c[i][a] * L->c[i][a]; }
            e += cc * fi;
        }
        double uu = 0.0, uF = 0.0;
        for (int a = 0; a < D; ++a) {
            u[(long)a * N + n] = (j[a] + 0.5 * Fn[a]) / rho[n];
            uu += u[(long)a * N + n] * u[(long)a * N + n];
            uF += u[(long)a * N + n] * Fn[a];
            F[(long)a * N + n] = Fn[a];
            Fsc[(long)a * N + n] = fs[a];
        }
        /* G2 = sum_i |c_i|^2 S_i: 2 u.F from F_i, 0 from H_i, and from P_i
         * -k cs2^2 |F^SC|^2 / (tau psi^2 G) (its only moment is the trace). */
        double G2 = 2.0 * uF;
        if (P->use_SC && P->use_P && psi[n] > 0.0) {
            double f2 = 0.0;
            for (int a = 0; a < D; ++a) f2 += fs[a] * fs[a];
            G2 += -P->k * s * s * f2 / ((P->tau_hat - 0.5) * psi[n] * psi[n] * G_SC);
        }
        theta[n] = (e - rho[n] * uu + 0.5 * G2) / (rho[n] * D * s);
    }
}

/* One step f_in -> f_out (Eq. 4.4 then streaming).  gfield: [D][N] acceleration or NULL. */
int or_step(const or_lattice* L, const or_params* P, const double* f_in, double* f_out, const double* gfield) {
    const long N = (long)P->nx * P->ny * P->nz;
    const int D = L->D, Q = L->Q;
    double* rho = malloc(sizeof(double) * N);
    double* th = malloc(sizeof(double) * N);
    double* psi = malloc(sizeof(double) * N);
    double* u = malloc(sizeof(double) * 3 * N);
    double* F = malloc(sizeof(double) * 3 * N);
    double* Fsc = malloc(sizeof(double) * 3 * N);
    double* gT = malloc(sizeof(double) * 3 * N);
    if (!rho || !th || !psi || !u || !F || !Fsc || !gT) {
        free(rho); free(th); free(psi); free(u); free(F); free(Fsc); free(gT);
        return -1;
    }
    or_macros(L, P, f_in, gfield, rho, u, th, F, psi, Fsc);
    if (P->use_H) {
        #pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            for (int a = 0; a < D; ++a) {
                int cp[3] = {0, 0, 0}, cm[3] = {0, 0, 0};
                cp[a] = 1; cm[a] = -1;
                gT[(long)a * N + n] = 0.5 * (th[nbr(P, n, cp)] - th[nbr(P, n, cm)]);
            }
        }
    }
    const double tau = P->tau_hat;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double feq[OR_MAXQ], SF[OR_MAXQ], SH[OR_MAXQ], SP[OR_MAXQ];
        double un[3] = {0, 0, 0}, Fn[3] = {0, 0, 0}, gn[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            un[a] = u[(long)a * N + n];
            Fn[a] = F[(long)a * N + n];
            fs[a] = Fsc[(long)a * N + n];
            if (P->use_H) gn[a] = gT[(long)a * N + n];
        }
        double theta_eq = P->thermal ? th[n] : 1.0;
        or_feq(L, P->feq_order, rho[n], un, theta_eq, feq);
        or_sources(L, P, rho[n], un, theta_eq, Fn, gn, fs, psi[n], SF, SH, SP);
        for (int i = 0; i < Q; ++i) {
            double S = SF[i];
            if (P->use_H) S += SH[i];
            if (P->use_SC && P->use_P) S += SP[i];
            double fi = f_in[(long)i * N + n];
            double fstar = fi - (fi - feq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * S;
            f_out[(long)i * N + nbr(P, n, L->c[i])] = fstar;
        }
    }
    free(rho); free(th); free(psi); free(u); free(F); free(Fsc); free(gT);
    return 0;
}

/* nsteps steps; f holds the state before and after, tmp is scratch of the same size. */
int or_run(const or_lattice* L, const or_params* P, double* f, double* tmp, const double* gfield, int nsteps) {
    const long N = (long)P->nx * P->ny * P->nz;
    for (int t = 0; t < nsteps; ++t) {
        if (or_step(L, P, f, tmp, gfield)) return -1;
        memcpy(f, tmp, sizeof(double) * (size_t)L->Q * N);
    }
    return 0;
}

/* Initial state f^_i = f^eq_i(rho, u, theta) with no non-equilibrium part. */
void or_init(const or_lattice* L, const or_params* P, const double* rho, const double* u,
             const double* theta, double* f) {
    const long N = (long)P->nx * P->ny * P->nz;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double feq[OR_MAXQ], un[3] = {0, 0, 0};
        for (int a = 0; a < L->D; ++a) un[a] = u[(long)a * N + n];
        or_feq(L, P->feq_order, rho[n], un, theta[n], feq);
        for (int i = 0; i < L->Q; ++i) f[(long)i * N + n] = feq[i];
    }
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

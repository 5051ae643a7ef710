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
 *   (The single-pass variant, lag = 1, takes grad theta and F^SC / P_i from
 *   the previous step's temperature and pseudopotential fields instead.)
 *   3. per node and velocity, the literal Table 2 polynomials:
 *        f^eq_i (Eq. 2.2 scaled), F_i (Eq. 3.3 scaled), H_i (Eq. 3.7
 *        scaled), P_i (Eq. 3.12 scaled); S_i = F_i + H_i + P_i.
 *   4. collision, Eq. 4.4:
 *        f*_i = f^_i - (f^_i - f^eq_i) / tau^ + (1 - 1 / (2 tau^)) S_i
 *   5. streaming: f^_i(x + c_i, t + 1) = f*_i(x), periodic in every axis.
 *   With walls (Sec. 4.3) the populations that arrive from beyond a wall are
 *   replaced first (or_wall_complete, Eqs. 4.7-4.8), and grad theta at the
 *   wall rows is a one-sided second-order difference into the fluid.
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
    int walls;          /* 0: periodic in y; 1: TMS walls below and above (Sec. 4.3) */
    int wall_rule;      /* 0: the reading of Eqs. 4.7-4.8 used; 1: Eq. 4.7 as printed */
    double wall_u[2][3];     /* velocity of the bottom (0) and top (1) wall */
    double wall_theta[2];    /* temperature of the bottom and top wall */
    int lag;            /* 1: neighbour fields (theta for grad theta, psi for F^SC and P_i)
                           of the previous step: the single-pass variant */
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
/* psi_field: the pseudopotential field F^SC and P_i use (NULL: psi of this
 * step's densities; the previous step's in the lagged variant). */
void or_macros_psi(const or_lattice* L, const or_params* P, const double* f, const double* gfield,
                   const double* psi_field, double* rho, double* u, double* theta, double* F, double* psi,
                   double* Fsc) {
    const long N = (long)P->nx * P->ny * P->nz;
    const int D = L->D, Q = L->Q;
    const double s = L->cs2;
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += f[(long)i * N + n];
        rho[n] = r;
        psi[n] = P->use_SC ? (psi_field ? psi_field[n] : or_psi(P, s, r)) : 0.0;
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

void or_macros(const or_lattice* L, const or_params* P, const double* f, const double* gfield,
               double* rho, double* u, double* theta, double* F, double* psi, double* Fsc) {
    or_macros_psi(L, P, f, gfield, NULL, rho, u, theta, F, psi, Fsc);
}

/* Tamm-Mott-Smith wall boundary (Sec. 4.3, Eqs. 4.7-4.8): walls below row 0
 * and above row ny - 1, periodic in x (and z).
 *
 * Geometry: rows 0 and ny - 1 are the wall nodes; the solid-liquid interface
 * lies half a cell inside them, at y = 1/2 and y = ny - 3/2, so the fluid
 * layer is H = ny - 2 high (Sec. 5.1: 56 rows, "actual height 54"; Sec. 5.3:
 * 102 rows, H = 100).
 *
 * After streaming, a node whose pull source x - c_i lies beyond the wall rows
 * has an unknown population i: the wall rows and the two rows next to each
 * (reach 3).  The periodic push of the step delivered there, in the slot of
 * the opposite direction ibar, the population f*_ibar(x) that left x across
 * the wall; this routine reads it and replaces the unknowns.
 *
 * wall_rule 0 (the reading used), at a node r rows from its wall node:
 *   f_i = f*_ibar(x) + s f^eq_i(rho_p, u_i, theta_i) - f^eq_ibar(rho_p, u_p, theta_p)
 * Eq. 4.7 with f_ibar the population that left x in the opposite direction
 * and the local state (rho_p, u_p, theta_p) the node's moments of the
 * previous step (the state that population relaxed toward): it comes back
 * with its non-equilibrium part, its equilibrium exchanged for one at the
 * wall's state.  u_i, theta_i: the wall's velocity and temperature
 * extrapolated linearly from the interface, through the first fluid row's
 * previous moments u_1, theta_1, to the point where population i turned back,
 * y = r - |c_iy| / 2 rows from the wall node.  s rescales the target density
 * so that the unknowns carry exactly the mass that left (sum_U f_i =
 * sum_U f*_ibar): the wall is impermeable.
 *
 * wall_rule 1 is Eqs. 4.7-4.8 as printed: the local moments are those of the
 * mixture of the known populations and f^eq_i(targets) for the unknowns
 * (Eq. 4.8, with the half-force shift), the targets are the wall's velocity
 * and temperature at the wall node and the previous moments at the fluid
 * nodes, and f_i = f_ibar + f^eq_i(target) - f^eq_i(local) with f_ibar the
 * post-streaming opposite population at x.  It carries almost none of a
 * moving wall's momentum into the fluid.
 * bcm holds the previous step's moments [rho, u_1..u_D, theta][N].
 */
static int or_opposite(const or_lattice* L, int i) {
    for (int j = 0; j < L->Q; ++j) {
        int same = 1;
        for (int a = 0; a < 3; ++a) same &= (L->c[j][a] == -L->c[i][a]);
        if (same) return j;
    }
    return -1;
}

/* Eqs. 4.7-4.8 as printed (wall_rule 1) at node n with unknown set unk. */
static void or_wall_printed(const or_lattice* L, const or_params* P, const double* f, double* fc,
                            const double* gfield, const double* bcm, long n, long r, int side,
                            const int* unk, const int* opp) {
    const long N = (long)P->nx * P->ny * P->nz;
    const int D = L->D, Q = L->Q;
    double rt = bcm[n], ut[3] = {0, 0, 0}, tt = bcm[(long)(1 + D) * N + n];
    for (int a = 0; a < D; ++a) ut[a] = bcm[(long)(1 + a) * N + n];
    if (r == 0) {
        for (int a = 0; a < D; ++a) ut[a] = P->wall_u[side][a];
        tt = P->wall_theta[side];
    }
    double feq_t[OR_MAXQ], feq_l[OR_MAXQ];
    or_feq(L, P->feq_order, rt, ut, P->thermal ? tt : 1.0, feq_t);
    double rl = 0.0, j[3] = {0, 0, 0}, e = 0.0;
    for (int i = 0; i < Q; ++i) {
        const double gi = unk[i] ? feq_t[i] : f[(long)i * N + n];
        double cc = 0.0;
        rl += gi;
        for (int a = 0; a < D; ++a) { j[a] += L->c[i][a] * gi; cc += (double)L->c[i][a] * L->c[i][a]; }
        e += cc * gi;
    }
    double ul[3] = {0, 0, 0}, uu = 0.0, uF = 0.0;
    for (int a = 0; a < D; ++a) {
        double ga = 0.0;
        if (P->use_force) ga = gfield ? gfield[(long)a * N + n] : P->g_uniform[a];
        const double Fa = rl * ga;
        ul[a] = (j[a] + 0.5 * Fa) / rl;
        uu += ul[a] * ul[a];
        uF += ul[a] * Fa;
    }
    const double tl = (e - rl * uu + uF) / (rl * D * L->cs2);
    or_feq(L, P->feq_order, rl, ul, P->thermal ? tl : 1.0, feq_l);
    for (int i = 0; i < Q; ++i)
        if (unk[i]) fc[(long)i * N + n] = f[(long)opp[i] * N + n] + feq_t[i] - feq_l[i];
}

void or_wall_complete(const or_lattice* L, const or_params* P, const double* f, double* fc,
                      const double* gfield, const double* bcm) {
    const long N = (long)P->nx * P->ny * P->nz;
    const long nx = P->nx, ny = P->ny;
    const int D = L->D, Q = L->Q;
    memcpy(fc, f, sizeof(double) * (size_t)Q * N);
    if (!P->walls) return;
    int opp[OR_MAXQ];
    for (int i = 0; i < Q; ++i) opp[i] = or_opposite(L, i);
    #pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        const long y = (n / nx) % ny;
        const int side = (y < ny / 2) ? 0 : 1;
        const long r = side == 0 ? y : ny - 1 - y;             /* rows from the wall node */
        int unk[OR_MAXQ], nu = 0;
        for (int i = 0; i < Q; ++i) {
            const long ys = y - L->c[i][1];
            unk[i] = (ys < 0 || ys >= ny);
            nu += unk[i];
        }
        if (!nu) continue;
        if (P->wall_rule == 1) {
            or_wall_printed(L, P, f, fc, gfield, bcm, n, r, side, unk, opp);
            continue;
        }
        /* previous moments of this node and of the first fluid row of its column */
        const long n1 = (n % nx) + nx * ((side == 0 ? 1 : ny - 2) + ny * (n / (nx * ny)));
        double up[3] = {0, 0, 0}, u1[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            up[a] = bcm[(long)(1 + a) * N + n];
            u1[a] = bcm[(long)(1 + a) * N + n1];
        }
        const double rp = bcm[n], tp = bcm[(long)(1 + D) * N + n], t1 = bcm[(long)(1 + D) * N + n1];
        const double* uw = P->wall_u[side];
        const double tw = P->wall_theta[side];
        double feq_p[OR_MAXQ];
        or_feq(L, P->feq_order, rp, up, P->thermal ? tp : 1.0, feq_p);
        double dep[OR_MAXQ], fw[OR_MAXQ], m_dep = 0.0, m_neq = 0.0, m_w = 0.0;
        for (int i = 0; i < Q; ++i) {
            if (!unk[i]) continue;
            const double turn = (double)r - 0.5 * fabs((double)L->c[i][1]);  /* turning point */
            const double wgt = (0.5 - turn) / 0.5;                           /* 0 at the interface */
            double ui[3] = {0, 0, 0}, fe[OR_MAXQ];
            for (int a = 0; a < D; ++a) ui[a] = uw[a] + wgt * (uw[a] - u1[a]);
            const double ti = tw + wgt * (tw - t1);
            or_feq(L, P->feq_order, rp, ui, P->thermal ? ti : 1.0, fe);
            fw[i] = fe[i];
            const int mc[3] = {-L->c[i][0], -L->c[i][1], -L->c[i][2]};
            dep[i] = f[(long)opp[i] * N + nbr(P, n, mc)];      /* f*_ibar(x), pushed to x - c_i */
            m_dep += dep[i];
            m_neq += dep[i] - feq_p[opp[i]];
            m_w += fw[i];
        }
        const double s = (m_dep - m_neq) / m_w;             /* sum_U f_i = sum_U f*_ibar */
        for (int i = 0; i < Q; ++i)
            if (unk[i]) fc[(long)i * N + n] = dep[i] + s * fw[i] - feq_p[opp[i]];
    }
}

/* One step f_in -> f_out (Eq. 4.4 then streaming).  gfield: [D][N] acceleration
 * or NULL.  With walls, bcm ([rho, u_1..u_D, theta][N]) holds the previous
 * step's moments on entry (the wall targets) and this step's on return.
 * With lag, lagf ([theta, psi][N]) holds the previous step's temperature and
 * pseudopotential on entry (the neighbour fields of this step) and this
 * step's on return. */
int or_step(const or_lattice* L, const or_params* P, const double* f_in, double* f_out, const double* gfield,
            double* bcm, double* lagf) {
    const long N = (long)P->nx * P->ny * P->nz;
    const int D = L->D, Q = L->Q;
    double* rho = malloc(sizeof(double) * N);
    double* th = malloc(sizeof(double) * N);
    double* psi = malloc(sizeof(double) * N);
    double* u = malloc(sizeof(double) * 3 * N);
    double* F = malloc(sizeof(double) * 3 * N);
    double* Fsc = malloc(sizeof(double) * 3 * N);
    double* gT = malloc(sizeof(double) * 3 * N);
    double* fc = P->walls ? malloc(sizeof(double) * (size_t)Q * N) : NULL;
    if (!rho || !th || !psi || !u || !F || !Fsc || !gT || (P->walls && (!fc || !bcm)) || (P->lag && !lagf)) {
        free(rho); free(th); free(psi); free(u); free(F); free(Fsc); free(gT); free(fc);
        return -1;
    }
    if (P->walls) {
        or_wall_complete(L, P, f_in, fc, gfield, bcm);
        f_in = fc;
    }
    or_macros_psi(L, P, f_in, gfield, P->lag ? lagf + N : NULL, rho, u, th, F, psi, Fsc);
    if (P->walls) {
        for (long n = 0; n < N; ++n) {
            bcm[n] = rho[n];
            for (int a = 0; a < D; ++a) bcm[(long)(1 + a) * N + n] = u[(long)a * N + n];
            bcm[(long)(1 + D) * N + n] = th[n];
        }
    }
    /* neighbour temperatures of grad theta: this step's, or the previous
     * step's in the lagged variant */
    const double* thn = P->lag ? lagf : th;
    if (P->use_H) {
        #pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            const long y = (n / P->nx) % P->ny;
            for (int a = 0; a < D; ++a) {
                int cp[3] = {0, 0, 0}, cm[3] = {0, 0, 0};
                cp[a] = 1; cm[a] = -1;
                if (P->walls && a == 1 && (y == 0 || y == P->ny - 1)) {
                    /* wall rows: one-sided second-order difference into the fluid */
                    const double sg = (y == 0) ? 1.0 : -1.0;
                    const long n1 = n + (long)sg * P->nx, n2 = n + 2 * (long)sg * P->nx;
                    gT[(long)a * N + n] = sg * (-3.0 * thn[n] + 4.0 * thn[n1] - thn[n2]) / 2.0;
                } else {
                    gT[(long)a * N + n] = 0.5 * (thn[nbr(P, n, cp)] - thn[nbr(P, n, cm)]);
                }
            }
        }
    }
    if (P->lag) {
        /* this step's temperature and pseudopotential: the next step's neighbour fields */
        #pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            lagf[n] = th[n];
            lagf[N + n] = P->use_SC ? or_psi(P, L->cs2, rho[n]) : 0.0;
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
    free(rho); free(th); free(psi); free(u); free(F); free(Fsc); free(gT); free(fc);
    return 0;
}

/* nsteps steps; f holds the state before and after, tmp is scratch of the same size. */
int or_run(const or_lattice* L, const or_params* P, double* f, double* tmp, const double* gfield, int nsteps,
           double* bcm, double* lagf) {
    const long N = (long)P->nx * P->ny * P->nz;
    for (int t = 0; t < nsteps; ++t) {
        if (or_step(L, P, f, tmp, gfield, bcm, lagf)) return -1;
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

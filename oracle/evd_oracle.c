/*
 * evd_oracle.c -- plain FP64 CPU oracle of the forced explicit
 * velocity-difference (EVD) multicomponent lattice Boltzmann step of
 * Lourenco, Constantino & Tavares, "Forcing mass transfer approach in
 * multicomponent miscible mixtures using the lattice Boltzmann method"
 * (Chem. Eng. Sci. 2025, arXiv 2504.07059).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Everything is IEEE double precision, compiled without FMA contraction
 * (-ffp-contract=off) and without fast-math.  The step follows the paper's
 * order (Sec. 2, after the interpolation figure): the stored state is the
 * post-stream distribution f_t; one step computes the moments, the cross
 * relaxation times, collides term by term, then streams by SCATTER (push):
 * every source population is split over its 1/3/9 destination nodes with the
 * second-order interpolation weights, and weight that would land on a solid
 * node is lumped back into the source node as App. A prescribes.
 *
 * Parity status of each function is stated at its definition.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXS 6
#define OR_MAXQ 19

typedef struct {
    int lattice;          /* 0 = D2Q9 (the paper's lattice), 1 = D3Q19 (extension) */
    int nx, ny, nz;       /* nodes; nz = 1 for D2Q9 */
    unsigned wall_mask;   /* bit 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+ : impermeable wall */
    int ns;               /* number of species, 1..OR_MAXS, molar masses non-decreasing */
    double M[OR_MAXS];    /* molar masses; species 0 is the lightest (c = 1)      */
    double D[OR_MAXS * OR_MAXS]; /* Maxwell-Stefan diffusivities, symmetric      */
    double tau1;          /* self relaxation time of the lightest species         */
    double g[3];          /* specific body force: F_i = rho_i g                   */
    int tau_mode;         /* 0: closed forms for ns<=3, 1: dense solve always     */
    unsigned flags;       /* corrective forcing terms of Eq. (improved_forcing_scheme):
                             bit 0 S_diff, bit 1 S_p, bit 2 S_rho; 0 = standard term */
} or_config;

#define OR_S_DIFF 1u
#define OR_S_P 2u
#define OR_S_RHO 4u

typedef struct {
    double rho[OR_MAXS];
    double ueq[OR_MAXS][3];
    double u[3];
    double rho_mix, n, p;
    double tau[OR_MAXS];
    double tau_x[OR_MAXS * OR_MAXS];
    double feq[OR_MAXS][OR_MAXQ];
    double f0[OR_MAXS][OR_MAXQ];
    double om_self[OR_MAXS][OR_MAXQ];
    double om_pair[OR_MAXS][OR_MAXS][OR_MAXQ]; /* Omega^{ij}_alpha for j != i */
    double S[OR_MAXS][OR_MAXQ];
    double theta[OR_MAXS][3];
} or_diag;

typedef struct {
    or_config cfg;
    int Q, Dm;
    long nsites;
    int e[OR_MAXQ][3];
    double w[OR_MAXQ];
    int opp[OR_MAXQ];
    double c[OR_MAXS], cs2[OR_MAXS], tau[OR_MAXS];
    double *f, *fs, *fn;  /* [ns][Q][nsites] */
    double* acc;          /* [3][nsites] per-node specific force added to g, or NULL */
    double* rho_field;    /* [ns][nsites] densities of f_t, for the gradient terms */
    long t;
} or_state;

/* ---------------------------------------------------------------- lattices
 * D2Q9 in the order of Eq. (discrete_velocity_DLS): 0 rest, 1..4 axis
 * directions at angles (alpha-1)pi/2, 5..8 diagonals at (alpha-5)pi/2+pi/4.
 * The weights are not printed in the paper; the standard isotropic set
 * (4/9, 1/9, 1/36) is the one for which c_s^2 = c^2/3.
 * D3Q19 (not in the paper): rest, 6 axis, 12 face diagonals, weights
 * 1/3, 1/18, 1/36, opposites in adjacent pairs.
 */
static const int E2[9][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},
                             {1,1,0},{-1,1,0},{-1,-1,0},{1,-1,0}};
static const int E3[19][3] = {{0,0,0},
    {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
    {1,1,0},{-1,-1,0},{1,-1,0},{-1,1,0},
    {1,0,1},{-1,0,-1},{1,0,-1},{-1,0,1},
    {0,1,1},{0,-1,-1},{0,1,-1},{0,-1,1}};

static int lattice_setup(int lattice, int e[OR_MAXQ][3], double w[OR_MAXQ], int opp[OR_MAXQ], int* Dm)
{
    int Q, a, b, k;
    if (lattice == 0) {
        Q = 9; *Dm = 2;
        for (a = 0; a < 9; ++a) {
            for (k = 0; k < 3; ++k) e[a][k] = E2[a][k];
            w[a] = (a == 0) ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else if (lattice == 1) {
        Q = 19; *Dm = 3;
        for (a = 0; a < 19; ++a) {
            for (k = 0; k < 3; ++k) e[a][k] = E3[a][k];
            w[a] = (a == 0) ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        }
    } else {
        return 0;
    }
    for (a = 0; a < Q; ++a) {
        opp[a] = -1;
        for (b = 0; b < Q; ++b)
            if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == -e[a][2]) opp[a] = b;
    }
    return Q;
}

int or_lattice_info(int lattice, int* e_out /*[Q*3]*/, double* w_out, int* opp_out)
{
    int e[OR_MAXQ][3], opp[OR_MAXQ], Dm, a, k;
    double w[OR_MAXQ];
    int Q = lattice_setup(lattice, e, w, opp, &Dm);
    if (!Q) return 0;
    for (a = 0; a < Q; ++a) {
        for (k = 0; k < 3; ++k) if (e_out) e_out[3 * a + k] = e[a][k];
        if (w_out) w_out[a] = w[a];
        if (opp_out) opp_out[a] = opp[a];
    }
    return Q;
}

/* ---------------------------------------------------------- species table
 * Eq. (speed_DLS): c_i / c_1 = c_{s,i} / c_{s,1} = sqrt(M_1 / M_i), c_1 = 1.
 * Equal viscosity nu_i = nu_1 with nu_i = (tau_i - dt/2) c_{s,i}^2 (Sec. 3,
 * below Eq. epecies_momentum_eq; Sec. 4 preamble) fixes tau_i from tau_1.
 */
static int species_setup(const or_config* cfg, double c[], double cs2[], double tau[])
{
    int i;
    const double M1 = cfg->M[0];
    if (cfg->ns < 1 || cfg->ns > OR_MAXS || !(cfg->tau1 > 0.5)) return 0;
    for (i = 0; i < cfg->ns; ++i) {
        if (!(cfg->M[i] > 0.0)) return 0;
        if (i > 0 && cfg->M[i] < cfg->M[i - 1]) return 0;
    }
    for (i = 0; i < cfg->ns; ++i) {
        c[i] = sqrt(M1 / cfg->M[i]);
        cs2[i] = c[i] * c[i] / 3.0;
        /* (tau_i - 1/2) cs2_i = (tau_1 - 1/2) cs2_1 */
        tau[i] = 0.5 + (cfg->tau1 - 0.5) * (cs2[0] / cs2[i]);
    }
    return 1;
}

/* ------------------------------------------------- cross relaxation times
 * Simplified tau_ij / D_ij relation, Eq. (relation_tauij_diff_coeff), one
 * equation per pair i<j (species labelled by increasing molar mass, as in the
 * paper):
 *   A_ij / tau_ij + (1/D_ij) sum_{s != i,j} rho_s / tau_sj = B_ij,
 *   A_ij = (rho_i + rho_j)/D_ij + 2 n^2 M_i M_j / (p dt),  B_ij = 2 rho/(D_ij dt),
 * with the ideal-mixture pressure p = n M_1 c_{s,1}^2 (Sec. 4.1).
 * Binary: Eq. (Luo&Girimaji_tau).  Ternary: the three closed forms printed in
 * Sec. 4.1.  Any N: Gaussian elimination of the same system in 1/tau_ij.
 * tau_out is [ns][ns], symmetric, diagonal set to 0.
 */
static int pair_index(int i, int j, int ns)
{
    /* position of pair (min,max) in the list (0,1),(0,2),...,(1,2),... */
    int a = i < j ? i : j, b = i < j ? j : i, k = 0, r, s;
    for (r = 0; r < ns; ++r)
        for (s = r + 1; s < ns; ++s) {
            if (r == a && s == b) return k;
            ++k;
        }
    return -1;
}

int or_tau_cross_dense(const or_config* cfg, const double* rho, double* tau_out)
{
    const int ns = cfg->ns;
    const int np = ns * (ns - 1) / 2;
    double A[15][16];
    double n = 0.0, rho_mix = 0.0, p;
    const double dt = 1.0, cs2_1 = 1.0 / 3.0;
    int i, j, s, r, col, piv, k;
    if (ns < 2) return 1;
    for (i = 0; i < ns; ++i) { n += rho[i] / cfg->M[i]; rho_mix += rho[i]; }
    p = n * cfg->M[0] * cs2_1;
    for (r = 0; r < np; ++r) for (col = 0; col <= np; ++col) A[r][col] = 0.0;
    for (i = 0; i < ns; ++i)
        for (j = i + 1; j < ns; ++j) {
            const double Dij = cfg->D[i * ns + j];
            r = pair_index(i, j, ns);
            A[r][r] += (rho[i] + rho[j]) / Dij + 2.0 * n * n * cfg->M[i] * cfg->M[j] / (p * dt);
            for (s = 0; s < ns; ++s) {
                if (s == i || s == j) continue;
                A[r][pair_index(s, j, ns)] += rho[s] / Dij;
            }
            A[r][np] = 2.0 * rho_mix / (Dij * dt);
        }
    /* Gaussian elimination with partial pivoting on the augmented matrix */
    for (col = 0; col < np; ++col) {
        piv = col;
        for (r = col + 1; r < np; ++r) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return 0;
        if (piv != col) for (k = 0; k <= np; ++k) { double tmp = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = tmp; }
        for (r = col + 1; r < np; ++r) {
            const double m = A[r][col] / A[col][col];
            for (k = col; k <= np; ++k) A[r][k] -= m * A[col][k];
        }
    }
    for (col = np - 1; col >= 0; --col) {
        double acc = A[col][np];
        for (k = col + 1; k < np; ++k) acc -= A[col][k] * A[k][np];
        A[col][np] = acc / A[col][col];   /* now holds X = 1/tau of this pair */
    }
    for (i = 0; i < ns; ++i)
        for (j = 0; j < ns; ++j)
            tau_out[i * ns + j] = (i == j) ? 0.0 : 1.0 / A[pair_index(i, j, ns)][np];
    return 1;
}

int or_tau_cross(const or_config* cfg, const double* rho, double* tau_out)
{
    const int ns = cfg->ns;
    const double dt = 1.0, cs2_1 = 1.0 / 3.0;
    double n = 0.0, rho_mix = 0.0, p;
    int i;
    if (ns < 2) return 1;
    if (cfg->tau_mode == 1 || ns > 3) return or_tau_cross_dense(cfg, rho, tau_out);
    for (i = 0; i < ns; ++i) { n += rho[i] / cfg->M[i]; rho_mix += rho[i]; }
    p = n * cfg->M[0] * cs2_1;
    for (i = 0; i < ns * ns; ++i) tau_out[i] = 0.0;
    if (ns == 2) {
        /* Eq. (Luo&Girimaji_tau) */
        const double t12 = dt / 2.0 + n * n * cfg->M[0] * cfg->M[1] / (p * rho_mix) * cfg->D[0 * 2 + 1];
        tau_out[0 * 2 + 1] = tau_out[1 * 2 + 0] = t12;
        return 1;
    } else {
        /* Sec. 4.1 ternary closed forms; paper labels 1,2,3 -> indices 0,1,2 */
        const double r1 = rho[0], r2 = rho[1], r3 = rho[2];
        const double D12 = cfg->D[0 * 3 + 1], D13 = cfg->D[0 * 3 + 2], D23 = cfg->D[1 * 3 + 2];
        const double M1 = cfg->M[0], M2 = cfg->M[1], M3 = cfg->M[2];
        const double A12 = (r1 + r2) / D12 + 2.0 * n * n * M1 * M2 / (p * dt);
        const double A13 = (r1 + r3) / D13 + 2.0 * n * n * M1 * M3 / (p * dt);
        const double A23 = (r2 + r3) / D23 + 2.0 * n * n * M2 * M3 / (p * dt);
        const double B12 = 2.0 * rho_mix / (D12 * dt);
        const double B13 = 2.0 * rho_mix / (D13 * dt);
        const double B23 = 2.0 * rho_mix / (D23 * dt);
        const double t23 = (A23 - r1 * r2 / (A13 * D13 * D23)) / (B23 - r1 * B13 / (A13 * D23));
        const double t12 = 1.0 / (B12 / A12 - r3 / (A12 * D12 * t23));
        const double t13 = 1.0 / (B13 / A13 - r2 / (A13 * D13 * t23));
        tau_out[0 * 3 + 1] = tau_out[1 * 3 + 0] = t12;
        tau_out[0 * 3 + 2] = tau_out[2 * 3 + 0] = t13;
        tau_out[1 * 3 + 2] = tau_out[2 * 3 + 1] = t23;
        return 1;
    }
}

/* Specific body force at node X: the uniform g of the configuration plus
 * the node's entry of the force field, when one is set (Sec. 4.2, Case II:
 * F_i(r) = rho_i omega^2 r is such a field). */
static void node_force(const or_state* st, long X, double a[3])
{
    int k;
    for (k = 0; k < 3; ++k) a[k] = st->cfg.g[k] + (st->acc ? st->acc[(long)k * st->nsites + X] : 0.0);
}

/* -------------------------------------------------------------- collision
 * One node, all species, term by term in the paper's notation:
 *   moments: Eq. (zeroth_order_moment), Eq. (first_order_moment_force),
 *            Eq. (Sirovich_mixture_density), Eq. (Sirovich_mixture_velocity)
 *   f^{i(eq)}: second-order equilibrium below Eq. (feqi0), mixture velocity u
 *   f^{i(0)}:  Eq. (feqi0)
 *   Omega^{ii}: Eq. (BGK_self_collision)
 *   Omega^{ij}: Eq. (Cross_collision_Sirovich), pair by pair
 *   S^i:        Eq. (CE_forcing_term_discretized), F_i = rho_i g
 *   update:     Eq. (LBE_forcing), f* = f + Omega^{ii} + sum_j Omega^{ij}
 *                                     + (1 - dt/(2 tau_i)) S^i
 * f and fstar are [ns][Q] for this node.  Returns 0 on a non-positive density.
 */
/* grad: NULL, or per node the gradients of the species densities [ns][3]
 * followed by the gradient of the mixture density [3], for S_p and S_rho. */
static int collide_node(const or_state* st, const double* f, double* fstar, or_diag* dg, const double* acc,
                        const double* grad)
{
    const or_config* cfg = &st->cfg;
    const int ns = cfg->ns, Q = st->Q;
    const double dt = 1.0;
    double rho[OR_MAXS] = {0}, ueq[OR_MAXS][3] = {{0}}, F[OR_MAXS][3] = {{0}}, u[3] = {0, 0, 0};
    double rho_mix = 0.0, tau_x[OR_MAXS * OR_MAXS];
    int i, j, a, k, l;

    for (i = 0; i < ns; ++i) {
        double mom[3] = {0, 0, 0};
        rho[i] = 0.0;
        for (a = 0; a < Q; ++a) {
            const double fa = f[i * Q + a];
            rho[i] += fa;
            for (k = 0; k < 3; ++k) mom[k] += st->c[i] * st->e[a][k] * fa;
        }
        if (!(rho[i] > 0.0)) return 0;
        for (k = 0; k < 3; ++k) {
            F[i][k] = rho[i] * acc[k];   /* F_i = rho_i (g + k(x)) */
            ueq[i][k] = mom[k] / rho[i] + F[i][k] * dt / (2.0 * rho[i]);
        }
        rho_mix += rho[i];
    }
    for (i = 0; i < ns; ++i)
        for (k = 0; k < 3; ++k) u[k] += (rho[i] / rho_mix) * ueq[i][k];
    if (!or_tau_cross(cfg, rho, tau_x)) return 0;

    for (i = 0; i < ns; ++i) {
        const double cs2 = st->cs2[i], tau_i = st->tau[i];
        /* corrective terms (Eq. improved_forcing_scheme): the vectors they
         * contract with [(e e - cs2 I)/cs2^2 . u] (S_diff: Theta_i dt/(2 tau_i
         * - dt); S_p, with a minus sign: grad(rho_i cs2)) and with
         * [(e e - cs2 I)/cs2 . u_i^eq] (S_rho: w_i grad rho, w_i = rho_i/rho) */
        double Xc[3] = {0, 0, 0}, Yc[3] = {0, 0, 0};
        if (cfg->flags & OR_S_DIFF)
            for (k = 0; k < 3; ++k) {
                double th = 0.0;
                for (j = 0; j < ns; ++j)
                    if (j != i) th += rho[i] * rho[j] / (rho_mix * tau_x[i * ns + j]) * (ueq[i][k] - ueq[j][k]);
                Xc[k] += dt / (2.0 * tau_i - dt) * th;
            }
        if ((cfg->flags & OR_S_P) && grad)
            for (k = 0; k < 3; ++k) Xc[k] -= cs2 * grad[i * 3 + k];
        if ((cfg->flags & OR_S_RHO) && grad)
            for (k = 0; k < 3; ++k) Yc[k] = (rho[i] / rho_mix) * grad[ns * 3 + k];
        for (a = 0; a < Q; ++a) {
            double ei[3], emu[3], eu = 0.0, usq = 0.0, proj = 0.0, feq, f0, om_self, om_cross = 0.0, S = 0.0;
            for (k = 0; k < 3; ++k) {
                ei[k] = st->c[i] * st->e[a][k];
                emu[k] = ei[k] - u[k];
                eu += ei[k] * u[k];
                usq += u[k] * u[k];
                proj += emu[k] * (ueq[i][k] - u[k]);
            }
            feq = st->w[a] * rho[i] * (1.0 + eu / cs2 + (eu * eu) / (2.0 * cs2 * cs2) - usq / (2.0 * cs2));
            f0 = (1.0 + proj / cs2) * feq;
            om_self = -(f[i * Q + a] - f0) / tau_i;
            for (j = 0; j < ns; ++j) {
                double dv = 0.0, om;
                if (j == i) continue;
                for (k = 0; k < 3; ++k) dv += emu[k] * (ueq[i][k] - ueq[j][k]);
                om = -(1.0 / tau_x[i * ns + j]) * (rho[j] / rho_mix) * (feq / cs2) * dv;
                om_cross += om;
                if (dg) dg->om_pair[i][j][a] = om;
            }
            for (k = 0; k < 3; ++k) {
                double v = ei[k] / cs2;
                for (l = 0; l < 3; ++l)
                    v += (ei[k] * ei[l] - cs2 * (k == l ? 1.0 : 0.0)) / (cs2 * cs2) * u[l];
                S += v * F[i][k];
            }
            if (cfg->flags) {
                double corr = 0.0;
                for (k = 0; k < 3; ++k)
                    for (l = 0; l < 3; ++l) {
                        const double t = ei[k] * ei[l] - cs2 * (k == l ? 1.0 : 0.0);
                        corr += t / (cs2 * cs2) * u[l] * Xc[k] + t / cs2 * ueq[i][l] * Yc[k];
                    }
                S += corr;
            }
            S *= st->w[a];
            fstar[i * Q + a] = f[i * Q + a] + om_self + om_cross + (1.0 - dt / (2.0 * tau_i)) * S;
            if (dg) {
                dg->feq[i][a] = feq;
                dg->f0[i][a] = f0;
                dg->om_self[i][a] = om_self;
                dg->S[i][a] = S;
            }
        }
    }
    if (dg) {
        for (i = 0; i < ns; ++i) {
            dg->rho[i] = rho[i];
            dg->tau[i] = st->tau[i];
            for (k = 0; k < 3; ++k) {
                dg->ueq[i][k] = ueq[i][k];
                dg->theta[i][k] = 0.0;
                for (j = 0; j < ns; ++j)
                    if (j != i) /* Eq. (CE_theta_definition) */
                        dg->theta[i][k] += rho[i] * rho[j] / (rho_mix * tau_x[i * ns + j]) * (ueq[i][k] - ueq[j][k]);
            }
        }
        for (k = 0; k < 3; ++k) dg->u[k] = u[k];
        dg->rho_mix = rho_mix;
        dg->n = 0.0;
        for (i = 0; i < ns; ++i) dg->n += rho[i] / cfg->M[i];
        dg->p = dg->n * cfg->M[0] / 3.0;
        for (i = 0; i < ns * ns; ++i) dg->tau_x[i] = tau_x[i];
    }
    return 1;
}

/* --------------------------------------------------------------- streaming
 * Second-order interpolation, Eq. (Second_order_spatial_interpolation), read
 * in scatter form: after collision the population f*_alpha(X) of species i
 * travels to the off-lattice point X + e^i_alpha dt and is shared among the
 * lattice nodes X + d, d in {-1,0,1}^D, with the tensor-product weight
 *   prod_k W(s_k; d_k),  W(s;0) = 1 - s^2,  W(s;+1) = s(1+s)/2,
 *                        W(s;-1) = -s(1-s)/2,  s_k = e^i_alpha,k dt,
 * which is the paper's node weighting with A..H the eight neighbours
 * (A +x, B +y, C -x, D -y, E (+,+), F (-,+), G (-,-), H (+,-)).
 * Periodic faces wrap.  Impermeable walls (App. A) sit half-way between the
 * last fluid node and the first solid one.  Weight that would reach a solid
 * node is kept at the source node: in the opposite direction when the
 * population heads into the crossed wall(s) (e . d_s > 0, d_s = the crossing
 * components of d) and in the same direction otherwise; this reproduces every
 * flat-wall equation of App. A.  At edges and corners the case e . d_s = 0,
 * on which the paper is silent, keeps the weight in the same direction.
 */
static double W1(double s, int d)
{
    if (d == 0) return 1.0 - s * s;
    if (d == 1) return s * (1.0 + s) / 2.0;
    return -s * (1.0 - s) / 2.0;
}

static void stream_plane(or_state* st, const double* src, double* dst, int i, int a);

/* The planes of species i in directions a and opp(a) scatter only into each
 * other (a crossed wall deposits into a or opp(a) at the source node), so
 * each such pair is one independent task; within a task the lower direction
 * goes first, as in a plain loop over directions, so every destination
 * receives its terms in the same order whether or not the tasks run in
 * parallel (an OpenMP build runs them on all host cores; the sums are
 * bitwise those of the serial build). */
static void stream_push(or_state* st, const double* src, double* dst)
{
    const or_config* cfg = &st->cfg;
    const int ns = cfg->ns, Q = st->Q;
    const long nsites = st->nsites;
    long task;
    memset(dst, 0, sizeof(double) * (size_t)ns * Q * nsites);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (task = 0; task < (long)ns * Q; ++task) {
        const int i = (int)(task / Q), a0 = (int)(task % Q);
        const int a1 = st->opp[a0];
        if (a1 < a0) continue;   /* streamed with its partner */
        stream_plane(st, src, dst, i, a0);
        if (a1 != a0) stream_plane(st, src, dst, i, a1);
    }
}

/* Scatter of the plane of species i, direction a (see stream_push). */
static void stream_plane(or_state* st, const double* src, double* dst, int i, int a)
{
    const or_config* cfg = &st->cfg;
    const int Q = st->Q, Dm = st->Dm;
    const int nn[3] = {cfg->nx, cfg->ny, cfg->nz};
    const long nsites = st->nsites;
    int k;
    long X;
    double s[3];
    for (k = 0; k < 3; ++k) s[k] = st->c[i] * st->e[a][k];
    for (X = 0; X < nsites; ++X) {
        const int xs[3] = {(int)(X % cfg->nx), (int)((X / cfg->nx) % cfg->ny),
                           (int)(X / ((long)cfg->nx * cfg->ny))};
        const double val = src[((long)i * Q + a) * nsites + X];
        int d[3];
        for (d[2] = (Dm == 3 ? -1 : 0); d[2] <= (Dm == 3 ? 1 : 0); ++d[2])
            for (d[1] = -1; d[1] <= 1; ++d[1])
                for (d[0] = -1; d[0] <= 1; ++d[0]) {
                    double wgt = 1.0;
                    int dest[3], crossed = 0, dot = 0;
                    for (k = 0; k < Dm; ++k) wgt *= W1(s[k], d[k]);
                    if (wgt == 0.0) continue;
                    for (k = 0; k < 3; ++k) {
                        dest[k] = xs[k] + d[k];
                        if (dest[k] < 0 || dest[k] >= nn[k]) {
                            const unsigned wall = (cfg->wall_mask >> (2 * k)) & 3u;
                            if (wall) {
                                crossed = 1;
                                dot += st->e[a][k] * d[k];
                            } else {
                                dest[k] = (dest[k] + nn[k]) % nn[k];
                            }
                        }
                    }
                    if (!crossed) {
                        const long Y = dest[0] + (long)cfg->nx * (dest[1] + (long)cfg->ny * dest[2]);
                        dst[((long)i * Q + a) * nsites + Y] += wgt * val;
                    } else {
                        const int b = (dot > 0) ? st->opp[a] : a;
                        dst[((long)i * Q + b) * nsites + X] += wgt * val;
                    }
                }
    }
}

/* ------------------------------------------------------------------ state */
or_state* or_create(const or_config* cfg)
{
    or_state* st;
    size_t n;
    int k;
    if (!cfg || cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return NULL;
    if (cfg->lattice == 0 && cfg->nz != 1) return NULL;
    for (k = 0; k < 3; ++k) {
        const unsigned wm = (cfg->wall_mask >> (2 * k)) & 3u;
        if (wm == 1u || wm == 2u) return NULL; /* a dimension is either periodic or walled on both ends */
    }
    if (cfg->lattice == 0 && (cfg->wall_mask & 0x30u)) return NULL;
    st = (or_state*)calloc(1, sizeof(or_state));
    if (!st) return NULL;
    st->cfg = *cfg;
    st->Q = lattice_setup(cfg->lattice, st->e, st->w, st->opp, &st->Dm);
    if (!st->Q || !species_setup(cfg, st->c, st->cs2, st->tau)) { free(st); return NULL; }
    st->nsites = (long)cfg->nx * cfg->ny * cfg->nz;
    n = (size_t)cfg->ns * st->Q * st->nsites;
    st->f = (double*)calloc(n, sizeof(double));
    st->fs = (double*)calloc(n, sizeof(double));
    st->fn = (double*)calloc(n, sizeof(double));
    if (!st->f || !st->fs || !st->fn) { free(st->f); free(st->fs); free(st->fn); free(st); return NULL; }
    return st;
}

void or_destroy(or_state* st)
{
    if (!st) return;
    free(st->f); free(st->fs); free(st->fn); free(st->acc); free(st->rho_field); free(st);
}

/* Per-node specific force field k(x), [3][nsites] (x fastest inside each
 * component), added to the uniform g: F_i(x) = rho_i (g + k(x)).  NULL
 * removes it.  Set it before or_init, whose initial velocities use it.
 * Returns 0 if memory runs out. */
int or_set_force_field(or_state* st, const double* k)
{
    if (!k) {
        free(st->acc);
        st->acc = NULL;
        return 1;
    }
    if (!st->acc) st->acc = (double*)malloc(sizeof(double) * 3 * (size_t)st->nsites);
    if (!st->acc) return 0;
    memcpy(st->acc, k, sizeof(double) * 3 * (size_t)st->nsites);
    return 1;
}

void or_species_info(const or_state* st, double* c, double* cs2, double* tau)
{
    int i;
    for (i = 0; i < st->cfg.ns; ++i) { c[i] = st->c[i]; cs2[i] = st->cs2[i]; tau[i] = st->tau[i]; }
}

/* Initial state (Sec. 4.1 and 4.2): rho_i = x_i M_i n, species and mixture
 * velocities zero, f = f^{(0)} of Eq. (feqi0) with the equilibrium velocity
 * replaced by u_i0 = u_i^eq - F_i dt/(2 rho_i) = -g dt/2 and u = 0.
 * x is [ns][nsites]; n is [nsites] or NULL for n = 1. */
int or_init(or_state* st, const double* x, const double* nfield)
{
    const or_config* cfg = &st->cfg;
    const int ns = cfg->ns, Q = st->Q;
    const long nsites = st->nsites;
    const double dt = 1.0;
    int i, a, k;
    long X;
    for (X = 0; X < nsites; ++X) {
        const double n = nfield ? nfield[X] : 1.0;
        for (i = 0; i < ns; ++i) {
            const double rho_i = x[(long)i * nsites + X] * cfg->M[i] * n;
            double ui0[3], a0[3];
            if (!(rho_i > 0.0)) return 0;
            node_force(st, X, a0);
            for (k = 0; k < 3; ++k) ui0[k] = 0.0 - rho_i * a0[k] * dt / (2.0 * rho_i);
            for (a = 0; a < Q; ++a) {
                /* u = 0: f^{eq} = w rho_i; f^{(0)} = [1 + e.(u_i0 - 0)/cs2] f^{eq} */
                double eu0 = 0.0;
                for (k = 0; k < 3; ++k) eu0 += st->c[i] * st->e[a][k] * ui0[k];
                st->f[((long)i * Q + a) * nsites + X] = (1.0 + eu0 / st->cs2[i]) * st->w[a] * rho_i;
            }
        }
    }
    st->t = 0;
    return 1;
}

void or_set_f(or_state* st, const double* f)
{
    memcpy(st->f, f, sizeof(double) * (size_t)st->cfg.ns * st->Q * st->nsites);
}

void or_get_f(const or_state* st, double* f)
{
    memcpy(f, st->f, sizeof(double) * (size_t)st->cfg.ns * st->Q * st->nsites);
}

long or_time(const or_state* st) { return st->t; }

/* One collision of every node into st->fs.  Returns 0 on failure. */
/* Isotropic lattice gradient of a node field phi at X (a reading: the paper
 * does not say how the gradients of Eq. improved_forcing_scheme are
 * discretised): grad phi = (1/cs0^2) sum_a w_a e_a phi(X + e_a) with the unit
 * lattice's weights and cs0^2 = 1/3.  A neighbour beyond an impermeable wall
 * takes the value at X (zero normal gradient); periodic faces wrap. */
static void lattice_grad(const or_state* st, const double* phi, long X, double g[3])
{
    const or_config* cfg = &st->cfg;
    const int ext[3] = {cfg->nx, cfg->ny, cfg->nz};
    const long stride[3] = {1, cfg->nx, (long)cfg->nx * cfg->ny};
    const int crd[3] = {(int)(X % cfg->nx), (int)((X / cfg->nx) % cfg->ny), (int)(X / stride[2])};
    int a, k;
    g[0] = g[1] = g[2] = 0.0;
    for (a = 0; a < st->Q; ++a) {
        long Y = 0;
        int solid = 0;
        for (k = 0; k < 3; ++k) {
            int c = crd[k] + st->e[a][k];
            if (c < 0 || c >= ext[k]) {
                if ((cfg->wall_mask >> (2 * k)) & 3u) solid = 1;
                c = (c + ext[k]) % ext[k];
            }
            Y += c * stride[k];
        }
        {
            const double v = solid ? phi[X] : phi[Y];
            for (k = 0; k < 3; ++k) g[k] += st->w[a] * st->e[a][k] * v;
        }
    }
    for (k = 0; k < 3; ++k) g[k] *= 3.0;
}

static int collide_all(or_state* st)
{
    const int ns = st->cfg.ns, Q = st->Q;
    const long nsites = st->nsites;
    double fn[OR_MAXS * OR_MAXQ] = {0}, fo[OR_MAXS * OR_MAXQ] = {0};
    double grad[(OR_MAXS + 1) * 3];
    const int need_grad = (st->cfg.flags & (OR_S_P | OR_S_RHO)) != 0;
    int i, a, ok = 1;
    long X;
    if (need_grad) {
        /* densities of f_t at every node first: rho_i, then the mixture */
        if (!st->rho_field) st->rho_field = (double*)malloc(sizeof(double) * (size_t)(ns + 1) * nsites);
        if (!st->rho_field) return 0;
        for (X = 0; X < nsites; ++X) {
            double r = 0.0;
            for (i = 0; i < ns; ++i) {
                double ri = 0.0;
                for (a = 0; a < Q; ++a) ri += st->f[((long)i * Q + a) * nsites + X];
                st->rho_field[(long)i * nsites + X] = ri;
                r += ri;
            }
            st->rho_field[(long)ns * nsites + X] = r;
        }
    }
    /* nodes collide independently (an OpenMP build runs them in parallel; a
     * failing node then stops nothing else, and the step reports failure) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) private(fn, fo, grad, i, a) reduction(&& : ok)
#endif
    for (X = 0; X < nsites; ++X) {
        for (i = 0; i < ns; ++i)
            for (a = 0; a < Q; ++a) fn[i * Q + a] = st->f[((long)i * Q + a) * nsites + X];
        if (need_grad)
            for (i = 0; i <= ns; ++i) lattice_grad(st, st->rho_field + (long)i * nsites, X, grad + i * 3);
        {
            double acc[3];
            node_force(st, X, acc);
            if (!collide_node(st, fn, fo, NULL, acc, need_grad ? grad : NULL)) ok = 0;
        }
        for (i = 0; i < ns; ++i)
            for (a = 0; a < Q; ++a) st->fs[((long)i * Q + a) * nsites + X] = fo[i * Q + a];
    }
    return ok;
}

/* nsteps full steps: collide, then stream.  Returns steps done. */
long or_step(or_state* st, long nsteps)
{
    long s;
    for (s = 0; s < nsteps; ++s) {
        double* tmp;
        if (!collide_all(st)) return s;
        stream_push(st, st->fs, st->fn);
        tmp = st->f; st->f = st->fn; st->fn = tmp;
        st->t += 1;
    }
    return nsteps;
}

/* Streaming alone: treats the current state as post-collision populations
 * and replaces it by the streamed (interpolated, wall-closed) result. */
void or_stream_only(or_state* st)
{
    double* tmp;
    stream_push(st, st->f, st->fn);
    tmp = st->f; st->f = st->fn; st->fn = tmp;
}

/* Collision alone on the current state (no streaming). */
int or_collide_only(or_state* st)
{
    double* tmp;
    if (!collide_all(st)) return 0;
    tmp = st->f; st->f = st->fs; st->fs = tmp;
    return 1;
}

/* One node through the collision, with every intermediate term returned. */
int or_collide_node(const or_state* st, const double* f, double* fstar, or_diag* dg)
{
    return collide_node(st, f, fstar, dg, st->cfg.g, NULL);
}

int or_diag_size(void) { return (int)sizeof(or_diag); }

/* Threads a step uses: the OpenMP team size of an OpenMP build, else 1. */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Observables of the current state f_t, per node:
 *   rho_i (Eq. zeroth_order_moment), x_i = rho_i/(n M_i) with n = sum rho_j/M_j,
 *   mixture velocity u (Eq. Sirovich_mixture_velocity, forced u_i^eq),
 *   species velocity u_i = u_i^eq - dt Theta_i/(2 rho_i) (Eq. CE_EQ83),
 *   and u_i^eq itself.  Layouts: x, rho [ns][nsites]; u [3][nsites];
 *   ui, ueq [ns][3][nsites].  Any output may be NULL. */
int or_observables(const or_state* st, double* x, double* rho, double* u, double* ui, double* ueq)
{
    const int ns = st->cfg.ns, Q = st->Q;
    const long nsites = st->nsites;
    double fn[OR_MAXS * OR_MAXQ] = {0}, fo[OR_MAXS * OR_MAXQ] = {0};
    or_diag dg;
    int i, a, k;
    long X;
    for (X = 0; X < nsites; ++X) {
        for (i = 0; i < ns; ++i)
            for (a = 0; a < Q; ++a) fn[i * Q + a] = st->f[((long)i * Q + a) * nsites + X];
        {
            double acc[3];
            node_force(st, X, acc);
            if (!collide_node(st, fn, fo, &dg, acc, NULL)) return 0;
        }
        for (i = 0; i < ns; ++i) {
            if (x) x[(long)i * nsites + X] = dg.rho[i] / (dg.n * st->cfg.M[i]);
            if (rho) rho[(long)i * nsites + X] = dg.rho[i];
            for (k = 0; k < 3; ++k) {
                if (ui) ui[((long)i * 3 + k) * nsites + X] = dg.ueq[i][k] - 1.0 * dg.theta[i][k] / (2.0 * dg.rho[i]);
                if (ueq) ueq[((long)i * 3 + k) * nsites + X] = dg.ueq[i][k];
            }
        }
        if (u) for (k = 0; k < 3; ++k) u[(long)k * nsites + X] = dg.u[k];
    }
    return 1;
}

/* Per-species total mass sum_x sum_alpha f, Kahan-compensated. */
void or_mass(const or_state* st, double* m)
{
    const int ns = st->cfg.ns, Q = st->Q;
    const long nsites = st->nsites;
    int i, a;
    long X;
    for (i = 0; i < ns; ++i) {
        double s = 0.0, comp = 0.0;
        for (a = 0; a < Q; ++a)
            for (X = 0; X < nsites; ++X) {
                const double y = st->f[((long)i * Q + a) * nsites + X] - comp;
                const double t = s + y;
                comp = (t - s) - y;
                s = t;
            }
        m[i] = s;
    }
}

// evd_adjoint.cu -- kernels of the discrete adjoint of the step (D2Q9, FP64).
//
// One step maps f*_{t-1} to f*_t = C(G f*_{t-1}; theta): G the gather with
// the interpolation and the App. A walls (linear), C the node-local
// collision, theta = (D_ij for i < j, g_x, g_y).  Reverse sweep:
//   lambda_t  = C_t^T lambda*_t,   dL/dtheta += (dC_t/dtheta)^T lambda*_t,
//   lambda*_{t-1} = G^T lambda_t.
// C_t^T is exact; G^T is written out by hand (the scatter of the gather's
// weights, including the lumped wall terms).
//
// The collision of Eq. (LBE_forcing) is f*_ia = omt_i f_ia + h_ia(m, theta):
// apart from the linear term omt_i f_ia (omt_i = 1 - 1/tau_i), it depends on
// the populations only through the node moments m = (rho_i, J_x,i, J_y,i),
// rho_i = sum_a f_ia and J_i = sum_a e_a f_ia (Eq. zeroth_order_moment,
// first_order_moment_force), a constant linear map m = P f.  Hence
//   C^T lambda* = omt . lambda* + P^T mu,   mu_m = lambda* . dh/dm_m.
// Two kernels form mu and the parameter partials:
//   k_adj_collide_rev (default): reverse mode written out by hand through the
//     collision, recomputed in double;
//   k_adj_collide (cross-check): the step's own collision templates in
//     forward-mode dual numbers, dh/dm_m = C s_m - omt . s_m for population
//     seeds s_m with P s_m = the unit vector of m, so the dual numbers carry
//     3 NS moment tangents (seeds on the rest and the axis populations) plus
//     the parameters, not one tangent per population.
#include <cuda_runtime.h>

#include "evd_device.cuh"
#include "evd_dual.cuh"   // after evd_device.cuh: ADL supplies fma / isfinite for Dual
#include "evd_internal.h"

namespace evd {

constexpr int ADJ_BLOCK = 64;

template <int NS>
struct AdjDim {
    static constexpr int NP = NS * (NS - 1) / 2 + 2;   // D_ij (i < j), g_x, g_y
    static constexpr int NM = NS * 3;                   // node moments rho_i, J_x,i, J_y,i
    static constexpr int N = NM + NP;                   // tangents: moments, then parameters
};

// Seed of population A for moment r (0: rho, 1: J_x, 2: J_y) of its species:
// the rest population carries rho, the two x-axis populations +-1/2 of J_x,
// the two y-axis ones +-1/2 of J_y, so that P s_r is the unit vector of r.
template <int A>
__device__ constexpr double moment_seed(int r)
{
    constexpr int ex = ev<0>(A, 0), ey = ev<0>(A, 1);
    if (ex == 0 && ey == 0) return r == 0 ? 1.0 : 0.0;
    if (ey == 0) return r == 1 ? 0.5 * ex : 0.0;
    if (ex == 0) return r == 2 ? 0.5 * ey : 0.0;
    return 0.0;
}

// The collision's constants as dual numbers with the parameter tangents
// seeded: iD_ij = 1/D_ij moves with D_ij (d iD / dD = -iD^2), g with itself.
template <int NS, int N>
__device__ void dual_params(const Params<double>& p, Params<Dual<N>>& q)
{
    q.nx = p.nx; q.ny = p.ny; q.nz = p.nz; q.nsites = p.nsites; q.pstride = p.pstride;
    for (int k = 0; k < 3; ++k) { q.wall[k] = p.wall[k]; q.g[k] = Dual<N>(p.g[k]); q.wl[k] = Dual<N>(p.wl[k]); }
    for (int i = 0; i < MAXS; ++i) {
        q.unit[i] = p.unit[i];
        q.c[i] = p.c[i]; q.inv_cs2[i] = p.inv_cs2[i]; q.c_inv_cs2[i] = p.c_inv_cs2[i];
        q.tau_inv[i] = p.tau_inv[i]; q.omt[i] = p.omt[i]; q.sfac[i] = p.sfac[i];
        q.Minv[i] = p.Minv[i]; q.M[i] = p.M[i]; q.rref[i] = 0.0;
        for (int j = 0; j < MAXS; ++j) { q.MM[i][j] = p.MM[i][j]; q.iD[i][j] = p.iD[i][j]; }
        for (int a = 0; a < 3; ++a) {
            q.w1[i][a] = p.w1[i][a]; q.ref[i][a] = 0.0; q.refc[i][a] = 0.0;
            for (int b = 0; b < 3; ++b) q.w2[i][a][b] = p.w2[i][a][b];
        }
    }
    q.kf = nullptr;
    q.flags = 0;
    q.rhof = nullptr;
    int m = AdjDim<NS>::NM;
    for (int i = 0; i < NS; ++i)
        for (int j = i + 1; j < NS; ++j, ++m) {
            const double di = -p.iD[i][j] * p.iD[i][j];
            q.iD[i][j].d[m] = di;
            q.iD[j][i].d[m] = di;
        }
    q.g[0].d[m] = 1.0;
    q.g[1].d[m + 1] = 1.0;
}

// Per-block partial sums of NP doubles into part[blockIdx.x * NP + m].
template <int NP>
__device__ void block_partial(const double (&v)[NP], double* __restrict__ part)
{
    __shared__ double sm[NP][ADJ_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        double x = v[m];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sm[m][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double t = 0.0;
        for (int w = 0; w < ADJ_BLOCK / 32; ++w) t += sm[threadIdx.x][w];
        part[(long long)blockIdx.x * NP + threadIdx.x] = t;
    }
}

// lambda_t = C_t^T lambda*_t at every node, and the parameter partials.
// fin: f*_{t-1} (gathered here into f_t) or, with raw, f_0 itself.
template <int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
k_adj_collide(const Params<double> p, const double* __restrict__ fin, int raw, const double* __restrict__ lam_star,
              double* __restrict__ lam_f, double* __restrict__ part)
{
    constexpr int N = AdjDim<NS>::N, NP = AdjDim<NS>::NP, NM = AdjDim<NS>::NM, Q = 9;
    __shared__ Params<Dual<N>> q;
    if (threadIdx.x == 0) dual_params<NS, N>(p, q);
    __syncthreads();
    const int node = blockIdx.x * ADJ_BLOCK + threadIdx.x;
    double gpart[NP];
    for (int m = 0; m < NP; ++m) gpart[m] = 0.0;
    if (node < p.nsites) {
        double f0[NS][Q];
        if (raw) {
            load_raw<0, NS, double, double>(p, fin, node, f0);
        } else {
            const Nbr nb = neighbours(p, node);
            gather_all<0, NS>(p, fin, node, nb, f0);
        }
        Dual<N> f[NS][Q];
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            for (int i = 0; i < NS; ++i) {
                f[i][A] = Dual<N>(f0[i][A]);
                for (int r = 0; r < 3; ++r) f[i][A].d[3 * i + r] = moment_seed<A>(r);
            }
        });
        NodeState<NS, Dual<N>> s;
        unsigned err = 0;
        Dual<N> gn[3] = {q.g[0], q.g[1], q.g[2]};
        moments<0, NS, false>(q, f, s, err, gn);
        collide<0, NS, false>(q, f, s, gn);
        double ls[NS][Q];
        for (int i = 0; i < NS; ++i)
            for (int a = 0; a < Q; ++a) ls[i][a] = lam_star[(long long)plane_of<0, NS>(i, a) * p.pstride + node];
        // mu_m = lambda* . (C s_m) - lambda* . (omt . s_m)
        double mu[NM];
        for (int m = 0; m < NM; ++m) {
            double acc = 0.0;
            for (int i = 0; i < NS; ++i)
                for (int a = 0; a < Q; ++a) acc += ls[i][a] * f[i][a].d[m];
            mu[m] = acc;
        }
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            for (int i = 0; i < NS; ++i)
                for (int r = 0; r < 3; ++r) mu[3 * i + r] -= p.omt[i] * moment_seed<A>(r) * ls[i][A];
        });
        // lambda_ia = omt_i lambda*_ia + mu_rho,i + e_a . mu_J,i
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr int ex = ev<0>(A, 0), ey = ev<0>(A, 1);
            for (int i = 0; i < NS; ++i)
                lam_f[(long long)plane_of<0, NS>(i, A) * p.pstride + node] =
                    p.omt[i] * ls[i][A] + mu[3 * i] + ex * mu[3 * i + 1] + ey * mu[3 * i + 2];
        });
        for (int m = 0; m < NP; ++m) {
            double acc = 0.0;
            for (int i = 0; i < NS; ++i)
                for (int a = 0; a < Q; ++a) acc += ls[i][a] * f[i][a].d[NM + m];
            gpart[m] = acc;
        }
    }
    block_partial<NP>(gpart, part);
}

// Position of species pair (i, j), i < j, in the order (0,1), (0,2), ..., (1,2), ...
__host__ __device__ constexpr int pair_pos(int i, int j, int ns) { return i * (2 * ns - i - 1) / 2 + (j - i - 1); }

// The rates X_ij = 1/tau_ij of the closed forms that moments() evaluates
// (Eq. Luo&Girimaji_tau, the Sec. 4.1 ternary forms of Eq.
// relation_tauij_diff_coeff), one per pair, as dual numbers whose K = NS +
// pairs tangents are rho_0..rho_{NS-1} and the pair values iD_ij = 1/D_ij.
template <int NS, int K>
__device__ __forceinline__ void cross_rates_dual(const Params<double>& p, const double (&rho)[NS],
                                                 Dual<K> (&X)[NS * (NS - 1) / 2])
{
    Dual<K> r[NS];
    Dual<K> rm(0.0), n(0.0);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        r[i] = Dual<K>(rho[i]);
        r[i].d[i] = 1.0;
        rm += r[i];
        n += r[i] * Dual<K>(p.Minv[i]);
    }
    auto iD = [&](int i, int j) {
        Dual<K> v(p.iD[i][j]);
        v.d[NS + pair_pos(i, j, NS)] = 1.0;
        return v;
    };
    if constexpr (NS == 2) {
        const Dual<K> d01 = iD(0, 1);
        const Dual<K> A12 = (r[0] + r[1]) * d01 + n * Dual<K>(p.MM[0][1]);
        X[0] = Dual<K>(2.0) * rm * d01 / A12;
    } else if constexpr (NS == 3) {
        const Dual<K> d01 = iD(0, 1), d02 = iD(0, 2), d12 = iD(1, 2);
        const Dual<K> A12 = (r[0] + r[1]) * d01 + n * Dual<K>(p.MM[0][1]);
        const Dual<K> A13 = (r[0] + r[2]) * d02 + n * Dual<K>(p.MM[0][2]);
        const Dual<K> A23 = (r[1] + r[2]) * d12 + n * Dual<K>(p.MM[1][2]);
        const Dual<K> two_rm = Dual<K>(2.0) * rm;
        const Dual<K> B12 = two_rm * d01, B13 = two_rm * d02, B23 = two_rm * d12;
        const Dual<K> rA13 = Dual<K>(1.0) / A13;
        const Dual<K> X23 = (B23 - r[0] * B13 * rA13 * d12) / (A23 - r[0] * r[1] * rA13 * d02 * d12);
        X[0] = (B12 - r[2] * X23 * d01) / A12;   // pair (0,1)
        X[1] = (B13 - r[1] * X23 * d02) * rA13;  // pair (0,2)
        X[2] = X23;                              // pair (1,2)
    }
}

// lambda_t = C_t^T lambda*_t and the parameter partials by reverse mode,
// written out by hand.  The collision is recomputed in double (moments, u,
// tau_ij, V_i, the per-species scalars of collide()), then phi = sum_ia
// lambda*_ia h_ia (h the collision minus its linear term omt f) is swept
// backwards to its gradient with respect to the node moments (rho_i, J_i)
// and the parameters; C^T lambda* = omt . lambda* + P^T (d phi / d m).  The
// only forward-mode piece is the small Jacobian of the closed-form tau_ij.
template <int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
k_adj_collide_rev(const Params<double> p, const double* __restrict__ fin, int raw,
                  const double* __restrict__ lam_star, double* __restrict__ lam_f, double* __restrict__ part)
{
    constexpr int NP = AdjDim<NS>::NP, Q = 9;
    constexpr int NPAIR = NS * (NS - 1) / 2, NPA = NPAIR > 0 ? NPAIR : 1, K = NS + NPAIR;
    const int node = blockIdx.x * ADJ_BLOCK + threadIdx.x;
    double gpart[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) gpart[m] = 0.0;
    if (node < p.nsites) {
        double f[NS][Q];
        if (raw) {
            load_raw<0, NS, double, double>(p, fin, node, f);
        } else {
            const Nbr nb = neighbours(p, node);
            gather_all<0, NS>(p, fin, node, nb, f);
        }
        double ls[NS][Q];
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int a = 0; a < Q; ++a) ls[i][a] = lam_star[(long long)plane_of<0, NS>(i, a) * p.pstride + node];
        const double g[2] = {p.g[0], p.g[1]};

        // ---- forward: the quantities of moments() and collide()
        double rho[NS], J[NS][2], rinv[NS], ueq[NS][2], u[2], Uv[2] = {0.0, 0.0}, rm = 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            double r = 0.0, jx = 0.0, jy = 0.0;
            static_for<0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                const double v = f[i][A];
                r += v;
                if constexpr (ev<0>(A, 0) == 1) jx += v;
                if constexpr (ev<0>(A, 0) == -1) jx -= v;
                if constexpr (ev<0>(A, 1) == 1) jy += v;
                if constexpr (ev<0>(A, 1) == -1) jy -= v;
            });
            rho[i] = r;
            J[i][0] = jx;
            J[i][1] = jy;
            rinv[i] = 1.0 / r;
#pragma unroll
            for (int k = 0; k < 2; ++k) ueq[i][k] = p.c[i] * J[i][k] * rinv[i] + 0.5 * g[k];
            rm += r;
        }
        const double rinv_m = 1.0 / rm;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int i = 0; i < NS; ++i) Uv[k] += rho[i] * ueq[i][k];
            u[k] = Uv[k] * rinv_m;
        }
        Dual<K> Xd[NPA] = {};
        if constexpr (NS >= 2) cross_rates_dual<NS, K>(p, rho, Xd);
        auto xr = [&](int i, int j) { return Xd[i < j ? pair_pos(i, j, NS) : pair_pos(j, i, NS)].v; };
        double P[NS][2];
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < NS; ++j)
                    if (j != i) acc += rho[j] * xr(i, j) * (ueq[i][k] - ueq[j][k]);
                P[i][k] = acc;   // V_i = P_i / rho
            }
        const double usq = u[0] * u[0] + u[1] * u[1];
        const double ug = u[0] * g[0] + u[1] * g[1];
        double av[NS][2], Bc[NS], U2[NS], sr[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            double ua = 0.0;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                av[i][k] = (ueq[i][k] - u[k]) * p.tau_inv[i] - P[i][k] * rinv_m;
                ua += u[k] * av[i][k];
            }
            Bc[i] = p.tau_inv[i] - p.inv_cs2[i] * ua;
            U2[i] = 1.0 - 0.5 * p.inv_cs2[i] * usq;
            sr[i] = rho[i] * p.inv_cs2[i] * p.sfac[i];
        }

        // ---- reverse: h_ia = feq B + S with feq = w rho_i (t1 (1 + t1/2) + U2_i),
        // B = c/cs2 e.av_i + Bc_i, S = w sr_i (c_i e.g (1 + t1) - u.g), t1 = c/cs2 e.u
        double u_bar[2] = {0.0, 0.0}, g_bar[2] = {0.0, 0.0}, ug_bar = 0.0;
        double av_bar[NS][2], Bc_bar[NS], U2_bar[NS], sr_bar[NS], rho_bar[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            av_bar[i][0] = av_bar[i][1] = 0.0;
            Bc_bar[i] = U2_bar[i] = sr_bar[i] = rho_bar[i] = 0.0;
        }
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr int C = wclass<0>(A);
            constexpr double ex = ev<0>(A, 0), ey = ev<0>(A, 1);
            const double eu = ex * u[0] + ey * u[1];
            const double eg = ex * g[0] + ey * g[1];
            double eu_bar = 0.0, eg_bar = 0.0;
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const double l = ls[i][A];
                const double ea = ex * av[i][0] + ey * av[i][1];
                const double t1 = p.c_inv_cs2[i] * eu;
                const double wr = p.wl[C] * rho[i];
                const double poly = t1 * (0.5 * t1 + 1.0) + U2[i];
                const double B = p.c_inv_cs2[i] * ea + Bc[i];
                const double Kf = p.wl[C] * sr[i];
                const double feq_bar = l * B, B_bar = l * wr * poly;
                av_bar[i][0] += B_bar * p.c_inv_cs2[i] * ex;
                av_bar[i][1] += B_bar * p.c_inv_cs2[i] * ey;
                Bc_bar[i] += B_bar;
                rho_bar[i] += feq_bar * poly * p.wl[C];
                U2_bar[i] += feq_bar * wr;
                sr_bar[i] += l * p.wl[C] * (p.c[i] * eg * (1.0 + t1) - ug);
                eg_bar += l * Kf * p.c[i] * (1.0 + t1);
                ug_bar -= l * Kf;
                const double t1_bar = feq_bar * wr * (t1 + 1.0) + l * Kf * p.c[i] * eg;
                eu_bar += t1_bar * p.c_inv_cs2[i];
            }
            u_bar[0] += eu_bar * ex;
            u_bar[1] += eu_bar * ey;
            g_bar[0] += eg_bar * ex;
            g_bar[1] += eg_bar * ey;
        });
        // per-species scalars: sr, U2, Bc (through u.av), av
        double usq_bar = 0.0, rinv_m_bar = 0.0, P_bar[NS][2], ueq_bar[NS][2];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            rho_bar[i] += sr_bar[i] * p.inv_cs2[i] * p.sfac[i];
            usq_bar -= 0.5 * p.inv_cs2[i] * U2_bar[i];
            const double ua_bar = -p.inv_cs2[i] * Bc_bar[i];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                u_bar[k] += ua_bar * av[i][k];
                av_bar[i][k] += ua_bar * u[k];
                ueq_bar[i][k] = av_bar[i][k] * p.tau_inv[i];
                u_bar[k] -= av_bar[i][k] * p.tau_inv[i];
                const double V_bar = -av_bar[i][k];   // av = ... - V, V = P / rho
                rinv_m_bar += V_bar * P[i][k];
                P_bar[i][k] = rinv_m * V_bar;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            u_bar[k] += 2.0 * usq_bar * u[k] + ug_bar * g[k];
            g_bar[k] += ug_bar * u[k];
        }
        // P_i = sum_{j != i} rho_j X_ij (u_i^eq - u_j^eq)
        double Xbar[NPA], iD_bar[NPA];
#pragma unroll
        for (int q = 0; q < NPA; ++q) Xbar[q] = iD_bar[q] = 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                if (j == i) continue;
                const double x = xr(i, j);
                const double pd = P_bar[i][0] * (ueq[i][0] - ueq[j][0]) + P_bar[i][1] * (ueq[i][1] - ueq[j][1]);
                rho_bar[j] += x * pd;
                Xbar[i < j ? pair_pos(i, j, NS) : pair_pos(j, i, NS)] += rho[j] * pd;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    ueq_bar[i][k] += rho[j] * x * P_bar[i][k];
                    ueq_bar[j][k] -= rho[j] * x * P_bar[i][k];
                }
            }
        if constexpr (NS >= 2) {
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
#pragma unroll
                for (int k = 0; k < NS; ++k) rho_bar[k] += Xbar[q] * Xd[q].d[k];
#pragma unroll
                for (int m = 0; m < NPAIR; ++m) iD_bar[m] += Xbar[q] * Xd[q].d[NS + m];
            }
        }
        // u = Uv / rho, Uv = sum rho_i u_i^eq
#pragma unroll
        for (int k = 0; k < 2; ++k) rinv_m_bar += u_bar[k] * Uv[k];
        const double Uv_bar[2] = {rinv_m * u_bar[0], rinv_m * u_bar[1]};
        const double rm_bar = -rinv_m * rinv_m * rinv_m_bar;
        // u_i^eq = c_i J_i / rho_i + g / 2
        double J_bar[NS][2];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            rho_bar[i] += Uv_bar[0] * ueq[i][0] + Uv_bar[1] * ueq[i][1] + rm_bar;
            double rinv_bar = 0.0;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                ueq_bar[i][k] += rho[i] * Uv_bar[k];
                J_bar[i][k] = p.c[i] * rinv[i] * ueq_bar[i][k];
                rinv_bar += p.c[i] * J[i][k] * ueq_bar[i][k];
                g_bar[k] += 0.5 * ueq_bar[i][k];
            }
            rho_bar[i] -= rinv[i] * rinv[i] * rinv_bar;
        }

        // ---- lambda_ia = omt_i lambda*_ia + rho_bar_i + e_a . J_bar_i
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr double ex = ev<0>(A, 0), ey = ev<0>(A, 1);
#pragma unroll
            for (int i = 0; i < NS; ++i)
                lam_f[(long long)plane_of<0, NS>(i, A) * p.pstride + node] =
                    p.omt[i] * ls[i][A] + rho_bar[i] + ex * J_bar[i][0] + ey * J_bar[i][1];
        });
        // parameters: dL/dD_ij = dL/d iD_ij * (-iD_ij^2)
        if constexpr (NS >= 2) {
#pragma unroll
            for (int i = 0; i < NS; ++i)
#pragma unroll
                for (int j = i + 1; j < NS; ++j)
                    gpart[pair_pos(i, j, NS)] = -iD_bar[pair_pos(i, j, NS)] * p.iD[i][j] * p.iD[i][j];
        }
        gpart[NP - 2] = g_bar[0];
        gpart[NP - 1] = g_bar[1];
    }
    block_partial<NP>(gpart, part);
}

// lambda*_{t-1} = G^T lambda_t: node X collects, for each direction, the
// gather weight with which every destination O = X - o read it, and the
// lumped weights with which X's own populations fed X (App. A).
template <int NS>
__global__ void __launch_bounds__(128)
k_adj_gather(const Params<double> p, const double* __restrict__ lam_f, double* __restrict__ lam_star)
{
    const int X = blockIdx.x * 128 + threadIdx.x;
    if (X >= p.nsites) return;
    const Nbr nb = neighbours(p, X);
    const int crd[2] = {X % p.nx, X / p.nx};
    const int ext[2] = {p.nx, p.ny};
    static_for<0, NS>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        static_for<0, 9>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr int ex = ev<0>(A, 0), ey = ev<0>(A, 1);
            const double* lp = lam_f + (long long)plane_of<0, NS>(I, A) * p.pstride;
            double acc = 0.0;
#pragma unroll
            for (int oy = (ey ? -1 : 0); oy <= (ey ? 1 : 0); ++oy)
#pragma unroll
                for (int ox = (ex ? -1 : 0); ox <= (ex ? 1 : 0); ++ox) {
                    const int o[2] = {ox, oy};
                    int c[2];
                    bool exists = true;
                    for (int k = 0; k < 2; ++k) {
                        c[k] = crd[k] - o[k];
                        if (c[k] < 0 || c[k] >= ext[k]) {
                            if (p.wall[k]) exists = false;
                            c[k] = (c[k] + ext[k]) % ext[k];
                        }
                    }
                    if (exists) acc += push_weight<0, A>(p, I, -ox, -oy, 0) * lp[c[0] + p.nx * c[1]];
                }
            if constexpr (ex != 0 || ey != 0) {
                if (nb.any_wall) {
                    constexpr int AB = opp<0>(A);
                    acc += lumped<0, A>(p, I, nb, true) * lp[X] +
                           lumped<0, A>(p, I, nb, false) * lam_f[(long long)plane_of<0, NS>(I, AB) * p.pstride + X];
                }
            }
            lam_star[(long long)plane_of<0, NS>(I, A) * p.pstride + X] = acc;
        });
    });
}

// lambda_N = (dx/df_N)^T dL/dx with f_N gathered from f*_{N-1}:
// x_i = rho_i / (n M_i), n = sum_j rho_j / M_j, the same for every direction.
template <int NS>
__global__ void __launch_bounds__(128)
k_adj_readout(const Params<double> p, const double* __restrict__ fin, const double* __restrict__ dldx,
              double* __restrict__ lam_f)
{
    const int node = blockIdx.x * 128 + threadIdx.x;
    if (node >= p.nsites) return;
    double f[NS][9];
    const Nbr nb = neighbours(p, node);
    gather_all<0, NS>(p, fin, node, nb, f);
    double rho[NS], n = 0.0;
    for (int i = 0; i < NS; ++i) {
        rho[i] = 0.0;
        for (int a = 0; a < 9; ++a) rho[i] += f[i][a];
        n += rho[i] * p.Minv[i];
    }
    for (int j = 0; j < NS; ++j) {
        double cj = 0.0;
        for (int i = 0; i < NS; ++i) {
            const double dxi = ((i == j) ? p.Minv[i] / n : 0.0) - rho[i] * p.Minv[i] * p.Minv[j] / (n * n);
            cj += dldx[(long long)i * p.nsites + node] * dxi;
        }
        for (int a = 0; a < 9; ++a) lam_f[(long long)plane_of<0, NS>(j, a) * p.pstride + node] = cj;
    }
}

// The initial populations f_0 = w rho_i (1 - e.g / (2 c_s^2)) depend on g:
// dL/dg_k += sum lambda_0 d f_0 / d g_k.  Partials of NP entries (only the
// two g entries non-zero).
template <int NS>
__global__ void __launch_bounds__(ADJ_BLOCK)
k_adj_init_g(const Params<double> p, const double* __restrict__ x0, const double* __restrict__ n0,
             const double* __restrict__ lam0, double* __restrict__ part)
{
    constexpr int NP = AdjDim<NS>::NP;
    const int node = blockIdx.x * ADJ_BLOCK + threadIdx.x;
    double gpart[NP];
    for (int m = 0; m < NP; ++m) gpart[m] = 0.0;
    if (node < p.nsites) {
        const double n = n0 ? n0[node] : 1.0;
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const double r = x0[(long long)I * p.nsites + node] * p.M[I] * n;
            static_for<0, 9>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                const double l = lam0[(long long)plane_of<0, NS>(I, A) * p.pstride + node];
                const double base = -0.5 * p.wl[wclass<0>(A)] * r * p.c_inv_cs2[I] * l;
                gpart[NP - 2] += base * ev<0>(A, 0);
                gpart[NP - 1] += base * ev<0>(A, 1);
            });
        });
    }
    block_partial<NP>(gpart, part);
}

// acc[m] += sum over blocks of part[b][m], in a fixed order.
__global__ void __launch_bounds__(32) k_adj_sum(const double* __restrict__ part, int nblocks, int np, double* acc)
{
    for (int m = threadIdx.x; m < np; m += 32) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(long long)b * np + m];
        acc[m] += s;
    }
}

#define EVD_ADJ_DISPATCH(KERNEL, GRID, BLK, ...)                                      \
    switch (h.ns) {                                                                   \
        case 1: KERNEL<1><<<GRID, BLK, 0, st>>>(__VA_ARGS__); break;                  \
        case 2: KERNEL<2><<<GRID, BLK, 0, st>>>(__VA_ARGS__); break;                  \
        case 3: KERNEL<3><<<GRID, BLK, 0, st>>>(__VA_ARGS__); break;                  \
        default: return cudaErrorInvalidValue;                                        \
    }

int AdjLaunch::nparams(int ns) { return ns * (ns - 1) / 2 + 2; }

int AdjLaunch::nblocks(const HostParams& h) { return (h.nsites + ADJ_BLOCK - 1) / ADJ_BLOCK; }

cudaError_t AdjLaunch::collide(const HostParams& h, const double* fin, bool raw, const double* lam_star,
                               double* lam_f, double* part, double* grad, bool dual, cudaStream_t st)
{
    const Params<double> p = to_params<double>(h);
    const int nb = nblocks(h);
    if (dual) {
        EVD_ADJ_DISPATCH(k_adj_collide, nb, ADJ_BLOCK, p, fin, raw ? 1 : 0, lam_star, lam_f, part)
    } else {
        EVD_ADJ_DISPATCH(k_adj_collide_rev, nb, ADJ_BLOCK, p, fin, raw ? 1 : 0, lam_star, lam_f, part)
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_sum<<<1, 32, 0, st>>>(part, nb, nparams(h.ns), grad);
    return cudaGetLastError();
}

cudaError_t AdjLaunch::gather_t(const HostParams& h, const double* lam_f, double* lam_star, cudaStream_t st)
{
    const Params<double> p = to_params<double>(h);
    EVD_ADJ_DISPATCH(k_adj_gather, (h.nsites + 127) / 128, 128, p, lam_f, lam_star)
    return cudaGetLastError();
}

cudaError_t AdjLaunch::readout(const HostParams& h, const double* fin, const double* dldx, double* lam_f,
                               cudaStream_t st)
{
    const Params<double> p = to_params<double>(h);
    EVD_ADJ_DISPATCH(k_adj_readout, (h.nsites + 127) / 128, 128, p, fin, dldx, lam_f)
    return cudaGetLastError();
}

cudaError_t AdjLaunch::init_g(const HostParams& h, const double* x0, const double* n0, const double* lam0,
                              double* part, double* grad, cudaStream_t st)
{
    const Params<double> p = to_params<double>(h);
    const int nb = nblocks(h);
    EVD_ADJ_DISPATCH(k_adj_init_g, nb, ADJ_BLOCK, p, x0, n0, lam0, part)
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_sum<<<1, 32, 0, st>>>(part, nb, nparams(h.ns), grad);
    return cudaGetLastError();
}

}  // namespace evd

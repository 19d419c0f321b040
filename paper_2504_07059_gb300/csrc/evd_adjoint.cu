// evd_adjoint.cu -- kernels of the discrete adjoint of the step (D2Q9, FP64).
//
// One step maps f*_{t-1} to f*_t = C(G f*_{t-1}; theta): G the gather with
// the interpolation and the App. A walls (linear), C the node-local
// collision, theta = (D_ij for i < j, g_x, g_y).  Reverse sweep:
//   lambda_t  = C_t^T lambda*_t,   dL/dtheta += (dC_t/dtheta)^T lambda*_t,
//   lambda*_{t-1} = G^T lambda_t.
// C_t^T is taken exactly from the Jacobian of the collision, obtained by
// running the collision templates in forward-mode dual numbers with one
// tangent per input population and per parameter; G^T is written out by hand
// (the scatter of the gather's weights, including the lumped wall terms).
#include <cuda_runtime.h>

#include "evd_device.cuh"
#include "evd_dual.cuh"   // after evd_device.cuh: ADL supplies fma / isfinite for Dual
#include "evd_internal.h"

namespace evd {

constexpr int ADJ_BLOCK = 64;

template <int NS>
struct AdjDim {
    static constexpr int NP = NS * (NS - 1) / 2 + 2;   // D_ij (i < j), g_x, g_y
    static constexpr int N = NS * 9 + NP;               // tangents: populations, then parameters
};

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
    int m = NS * 9;
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
    constexpr int N = AdjDim<NS>::N, NP = AdjDim<NS>::NP, Q = 9;
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
        for (int i = 0; i < NS; ++i)
            for (int a = 0; a < Q; ++a) {
                f[i][a] = Dual<N>(f0[i][a]);
                f[i][a].d[i * Q + a] = 1.0;
            }
        NodeState<NS, Dual<N>> s;
        unsigned err = 0;
        Dual<N> gn[3] = {q.g[0], q.g[1], q.g[2]};
        moments<0, NS, false>(q, f, s, err, gn);
        collide<0, NS, false>(q, f, s, gn);
        double ls[NS][Q];
        for (int i = 0; i < NS; ++i)
            for (int a = 0; a < Q; ++a) ls[i][a] = lam_star[(long long)plane_of<0, NS>(i, a) * p.pstride + node];
        for (int k = 0; k < NS * Q; ++k) {
            double acc = 0.0;
            for (int i = 0; i < NS; ++i)
                for (int a = 0; a < Q; ++a) acc += ls[i][a] * f[i][a].d[k];
            lam_f[(long long)k * p.pstride + node] = acc;   // D2Q9 planes are i * 9 + a
        }
        for (int m = 0; m < NP; ++m) {
            double acc = 0.0;
            for (int i = 0; i < NS; ++i)
                for (int a = 0; a < Q; ++a) acc += ls[i][a] * f[i][a].d[NS * Q + m];
            gpart[m] = acc;
        }
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
                               double* lam_f, double* part, double* grad, cudaStream_t st)
{
    const Params<double> p = to_params<double>(h);
    const int nb = nblocks(h);
    EVD_ADJ_DISPATCH(k_adj_collide, nb, ADJ_BLOCK, p, fin, raw ? 1 : 0, lam_star, lam_f, part)
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

// evd_batch_kernels.cuh -- kernels of the batched step: every member of a
// batch advanced by the same per-node gather, moments, tau_ij and collision
// as the single-lattice general step (evd_device.cuh), over a work list of
// (member, site range) items.
#pragma once

#include "evd_device.cuh"

namespace evd {

// Per-item block sum of NS doubles, written to out[0..NS-1] by thread 0's
// warp in a fixed order (reproducible).
template <int NS>
__device__ __forceinline__ void block_sum(const double (&v)[NS], double* __restrict__ out)
{
    __shared__ double sm[NS][BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        double x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) sm[i][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < BLOCK / 32; ++w) t += sm[threadIdx.x][w];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// The member's constants into shared memory (all threads; the caller
// synchronises before the first use).
template <typename T>
__device__ __forceinline__ void load_params(Params<T>& dst, const Params<T>* __restrict__ src)
{
    static_assert(sizeof(Params<T>) % 4 == 0, "Params must be a whole number of words");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Params<T>) / 4); k += BLOCK) d[k] = __ldg(s + k);
}

// One time step of one work item: sites [node0, node0 + count) of a member
// whose populations start at fin / fout (the single-lattice step's node
// code, dithered rounding included).  Not inlined: it runs once per item,
// and three inlined species counts per kernel make D3Q19 compile very slowly.
template <int LAT, int NS, typename S, typename T>
__device__ __noinline__ void item_step(const Params<T>& p, const S* __restrict__ fin, S* __restrict__ fout,
                                          int node0, int count, double* __restrict__ part, unsigned& err,
                                          int flags, const double* __restrict__ corr)
{
    double m[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) m[i] = 0.0;
    for (int node = node0 + threadIdx.x; node < node0 + count; node += BLOCK) {
        NodeState<NS, T> s;
        step_node<LAT, NS>(p, fin, fout, node, corr, s, err);
#pragma unroll
        for (int i = 0; i < NS; ++i) m[i] += (double)s.rho[i];
    }
    if (flags & F_MASS) block_sum<NS>(m, part);
}

// One step of the whole batch: CTAs loop over the work items (persistent
// when the grid is smaller than the item count).  The step waits on global
// loads of the stencil, so residency matters more than registers: six CTAs
// per SM (at most 85 registers) measured fastest on the D2Q9 tube sweep.
template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(BLOCK, 6)
k_step_batch(const BatchItem* __restrict__ items, int n_items, const Params<T>* __restrict__ params,
             const MemberInfo* __restrict__ info, const S* __restrict__ fin, S* __restrict__ fout,
             double* __restrict__ part, unsigned* __restrict__ err_flag, int flags,
             const double* __restrict__ corr, unsigned* __restrict__ seed)
{
    __shared__ Params<T> sp;
    unsigned err = 0;
    // reduced storage: the step's seed of the dithered rounding, from the
    // device step counter seed[0] (read before this CTA counts itself done)
    const unsigned step_seed = seed ? (unsigned)((unsigned long long)(*(volatile unsigned*)seed + 1u) * 2654435761ull) | 1u : 0u;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem w = items[it];
        const long long off = info[w.member].foff;
        __syncthreads();   // the previous item is done with sp
        load_params(sp, params + w.member);
        if (seed && threadIdx.x == 0) sp.seed = step_seed;
        __syncthreads();
        const double* c = corr ? corr + (long long)w.member * MAXS : nullptr;
        double* pt = part + (long long)it * MAXS;
        switch (w.ns) {
            case 1: item_step<LAT, 1>(sp, fin + off, fout + off, w.node0, w.count, pt, err, flags, c); break;
            case 2: item_step<LAT, 2>(sp, fin + off, fout + off, w.node0, w.count, pt, err, flags, c); break;
            default: item_step<LAT, 3>(sp, fin + off, fout + off, w.node0, w.count, pt, err, flags, c); break;
        }
    }
    if (err) atomicOr(err_flag, err);
    if (seed) {   // the last CTA to finish advances the step counter for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(seed + 1, 1u) == gridDim.x - 1) {
                seed[1] = 0u;
                seed[0] += 1u;
                __threadfence();
            }
        }
    }
}

// Observables of one work item (as k_readout), written into the
// concatenated field arrays at the member's offsets.
template <int LAT, int NS, typename S, typename T>
__device__ __noinline__ void item_readout(const Params<T>& p, const MemberInfo& mi, const S* __restrict__ fin,
                                             int node0, int count, int flags, double* __restrict__ x,
                                             double* __restrict__ rho, double* __restrict__ u,
                                             double* __restrict__ ui, double* __restrict__ part, unsigned& err,
                                             const double* __restrict__ corr)
{
    constexpr int Q = Lat<LAT>::Q, D = Lat<LAT>::D;
    const long long n = mi.sites;
    double m[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) m[i] = 0.0;
    for (int node = node0 + threadIdx.x; node < node0 + count; node += BLOCK) {
        T f[NS][Q];
        T gn[3];   // specific body force at this node
        node_force(p, node, gn);
        NodeState<NS, T> s;
        T R0[NS];
        node_base<LAT, NS>(p, fin, node, R0);
        if (flags & F_RAW) {
            load_raw<LAT, NS>(p, fin, node, f);
        } else {
            const Nbr nb = neighbours(p, node);
            gather_all<LAT, NS>(p, fin, node, nb, R0, f);
            if (corr) add_correction<LAT, NS>(p, corr, f, R0);
        }
        moments<LAT, NS, dev_arith<S>()>(p, f, s, err, gn, R0);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            if (x) x[mi.xoff + i * n + node] = (double)(s.rho[i] * p.Minv[i]) / (double)s.n;
            if (rho) rho[mi.xoff + i * n + node] = (double)s.rho[i];
#pragma unroll
            for (int k = 0; k < D; ++k)   // u_i = u_i^eq - Theta_i/(2 rho_i), Eq. (CE_EQ83)
                if (ui) ui[mi.uioff + (i * D + k) * n + node] = (double)(s.ueq[i][k] - (T)0.5 * s.V[i][k]);
            m[i] += (double)s.rho[i];
        }
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (u) u[mi.uoff + k * n + node] = (double)s.u[k];
    }
    block_sum<NS>(m, part);
}

template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_readout_batch(const BatchItem* __restrict__ items, int n_items, const Params<T>* __restrict__ params,
                const MemberInfo* __restrict__ info, const S* __restrict__ fin, int flags,
                double* __restrict__ x, double* __restrict__ rho, double* __restrict__ u,
                double* __restrict__ ui, double* __restrict__ part, unsigned* __restrict__ err_flag,
                const double* __restrict__ corr)
{
    __shared__ Params<T> sp;
    unsigned err = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem w = items[it];
        const MemberInfo mi = info[w.member];
        __syncthreads();
        load_params(sp, params + w.member);
        __syncthreads();
        const double* c = corr ? corr + (long long)w.member * MAXS : nullptr;
        double* pt = part + (long long)it * MAXS;
        const S* f = fin + mi.foff;
        switch (w.ns) {
            case 1: item_readout<LAT, 1>(sp, mi, f, w.node0, w.count, flags, x, rho, u, ui, pt, err, c); break;
            case 2: item_readout<LAT, 2>(sp, mi, f, w.node0, w.count, flags, x, rho, u, ui, pt, err, c); break;
            default: item_readout<LAT, 3>(sp, mi, f, w.node0, w.count, flags, x, rho, u, ui, pt, err, c); break;
        }
    }
    if (err) atomicOr(err_flag, err);
}

// Initial state of one work item (as k_init from mole fractions).
template <int LAT, int NS, typename S, typename T>
__device__ __noinline__ void item_init(const Params<T>& p, const MemberInfo& mi, const double* __restrict__ xf,
                                          const double* __restrict__ nf, S* __restrict__ fprev,
                                          S* __restrict__ fcur, int node0, int count, double* __restrict__ part,
                                          unsigned& err)
{
    constexpr int Q = Lat<LAT>::Q;
    const long long n = mi.sites;
    double m[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) m[i] = 0.0;
    for (int node = node0 + threadIdx.x; node < node0 + count; node += BLOCK) {
        T f[NS][Q];
        T gn[3];   // specific body force at this node
        node_force(p, node, gn);
        NodeState<NS, T> s;
        const T nn = nf ? (T)nf[mi.soff + node] : (T)1;
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            const T r = (T)xf[mi.xoff + I * n + node] * p.M[I] * nn;
            static_for<0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                const T eg = edot<LAT, A>(gn);
                f[I][A] = p.wl[wclass<LAT>(A)] * r * ((T)1 - (T)0.5 * p.c_inv_cs2[I] * eg);
            });
        });
        T R0[NS];
        to_deviations<LAT, NS, S>(p, f, R0);
        moments<LAT, NS, dev_arith<S>()>(p, f, s, err, gn, R0);
        store_all<LAT, NS>(p, fprev, node, f, s.rho, R0);
        collide<LAT, NS, dev_arith<S>(), false, Codec<S>::NODE>(p, f, s, gn);
        store_all<LAT, NS>(p, fcur, node, f, s.rho, R0);
#pragma unroll
        for (int i = 0; i < NS; ++i) m[i] += (double)s.rho[i];
    }
    block_sum<NS>(m, part);
}

template <int LAT, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_init_batch(const BatchItem* __restrict__ items, int n_items, const Params<T>* __restrict__ params,
             const MemberInfo* __restrict__ info, const double* __restrict__ xf, const double* __restrict__ nf,
             S* __restrict__ fprev, S* __restrict__ fcur, double* __restrict__ part,
             unsigned* __restrict__ err_flag)
{
    __shared__ Params<T> sp;
    unsigned err = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem w = items[it];
        const MemberInfo mi = info[w.member];
        __syncthreads();
        load_params(sp, params + w.member);
        __syncthreads();
        double* pt = part + (long long)it * MAXS;
        S* fp = fprev + mi.foff;
        S* fc = fcur + mi.foff;
        switch (w.ns) {
            case 1: item_init<LAT, 1>(sp, mi, xf, nf, fp, fc, w.node0, w.count, pt, err); break;
            case 2: item_init<LAT, 2>(sp, mi, xf, nf, fp, fc, w.node0, w.count, pt, err); break;
            default: item_init<LAT, 3>(sp, mi, xf, nf, fp, fc, w.node0, w.count, pt, err); break;
        }
    }
    if (err) atomicOr(err_flag, err);
}

template <int LAT, typename S, typename T>
cudaError_t batch_step(const BatchArgs& a, const void* fin, void* fout, double* part, unsigned* err, int flags,
                       const double* corr, cudaStream_t st)
{
    if (a.n_items == 0) return cudaSuccess;
    k_step_batch<LAT, S, T><<<a.grid, BLOCK, 0, st>>>(a.items, a.n_items, (const Params<T>*)a.params, a.info,
                                                      (const S*)fin, (S*)fout, part, err, flags, corr, a.seed);
    return cudaGetLastError();
}

template <int LAT, typename S, typename T>
cudaError_t batch_readout(const BatchArgs& a, const void* fin, int flags, double* x, double* rho, double* u,
                          double* ui, double* part, unsigned* err, const double* corr, cudaStream_t st)
{
    if (a.n_items == 0) return cudaSuccess;
    k_readout_batch<LAT, S, T><<<a.grid, BLOCK, 0, st>>>(a.items, a.n_items, (const Params<T>*)a.params, a.info,
                                                         (const S*)fin, flags, x, rho, u, ui, part, err, corr);
    return cudaGetLastError();
}

template <int LAT, typename S, typename T>
cudaError_t batch_init(const BatchArgs& a, const double* x, const double* n, void* fprev, void* fcur, double* part,
                       unsigned* err, cudaStream_t st)
{
    if (a.n_items == 0) return cudaSuccess;
    k_init_batch<LAT, S, T><<<a.grid, BLOCK, 0, st>>>(a.items, a.n_items, (const Params<T>*)a.params, a.info, x, n,
                                                      (S*)fprev, (S*)fcur, part, err);
    return cudaGetLastError();
}

}  // namespace evd

#define EVD_DEFINE_BATCH_LAUNCHERS(PREC, LAT, S, T)                                                         \
    namespace evd {                                                                                     \
    template <>                                                                                         \
    cudaError_t BatchLaunch<PREC, LAT>::step(const BatchArgs& a, const void* fin, void* fout, double* part, \
                                             unsigned* err, int flags, const double* corr, cudaStream_t st) \
    {                                                                                                   \
        return batch_step<LAT, S, T>(a, fin, fout, part, err, flags, corr, st);                         \
    }                                                                                                   \
    template <>                                                                                         \
    cudaError_t BatchLaunch<PREC, LAT>::readout(const BatchArgs& a, const void* fin, int flags, double* x,  \
                                                double* rho, double* u, double* ui, double* part,       \
                                                unsigned* err, const double* corr, cudaStream_t st)     \
    {                                                                                                   \
        return batch_readout<LAT, S, T>(a, fin, flags, x, rho, u, ui, part, err, corr, st);             \
    }                                                                                                   \
    template <>                                                                                         \
    cudaError_t BatchLaunch<PREC, LAT>::init(const BatchArgs& a, const double* x, const double* n,          \
                                             void* fprev, void* fcur, double* part, unsigned* err,      \
                                             cudaStream_t st)                                           \
    {                                                                                                   \
        return batch_init<LAT, S, T>(a, x, n, fprev, fcur, part, err, st);                              \
    }                                                                                                   \
    }

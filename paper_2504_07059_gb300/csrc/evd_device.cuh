// evd_device.cuh -- device code of the fused EVD lattice Boltzmann step.
//
// One thread owns one lattice node and all of its species: the cross
// collision couples the species at a node, so every population of the node
// must be in registers before the collision.  The step is the "pull" form of
// the paper's time step: the stored buffer holds post-collision populations
// f*_{t-1}; a launch gathers them with the second-order interpolation of
// Eq. (Second_order_spatial_interpolation) (plus the App. A wall terms at
// wall-adjacent nodes) into f_t, computes the moments, the cross relaxation
// times and the collision of Eq. (LBE_forcing), and writes f*_t.
//
// Layout in HBM: structure of arrays, one plane per (species, direction) at
// element offset plane_of(i, a) * pstride, x fastest inside a plane, pstride
// rounded up to 64 elements so every plane starts 128-byte aligned.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "evd_internal.h"

namespace evd {

constexpr int BLOCK = 128;

enum : int { F_MASS = 1, F_RAW = 2 };          // kernel flags
enum : unsigned { ERR_RHO = 1u, ERR_TAU = 2u };  // device error bits

template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------- lattices
template <int LAT> struct Lat;
template <> struct Lat<0> { static constexpr int Q = 9, D = 2; };
template <> struct Lat<1> { static constexpr int Q = 19, D = 3; };

// Unit direction vectors; D2Q9 in the order of Eq. (discrete_velocity_DLS).
template <int LAT>
__host__ __device__ constexpr int ev(int a, int k)
{
    if (LAT == 0) {
        constexpr int E[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return E[a][k];
    } else {
        constexpr int E[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return E[a][k];
    }
}

template <int LAT>
__host__ __device__ constexpr int opp(int a)
{
    int b = 0;
    for (int c = 0; c < Lat<LAT>::Q; ++c)
        if (ev<LAT>(c, 0) == -ev<LAT>(a, 0) && ev<LAT>(c, 1) == -ev<LAT>(a, 1) &&
            ev<LAT>(c, 2) == -ev<LAT>(a, 2))
            b = c;
    return b;
}

// the first direction whose component d is non-zero (where a sum over that
// component starts), -1 if none
template <int LAT>
__host__ __device__ constexpr int first_dir(int d)
{
    for (int a = 0; a < Lat<LAT>::Q; ++a)
        if (ev<LAT>(a, d) != 0) return a;
    return -1;
}

// weight class = number of non-zero components: 0 rest, 1 axis, 2 diagonal
template <int LAT>
__host__ __device__ constexpr int wclass(int a)
{
    return (ev<LAT>(a, 0) != 0) + (ev<LAT>(a, 1) != 0) + (ev<LAT>(a, 2) != 0);
}

// Storage order of the population planes.  D2Q9: plane = i*9 + a.  D3Q19:
// directions are grouped by the dimensions they move in, G0 {0}, G1 {5,6},
// G2 {1,2}, G3 {11..14}, G4 {3,4}, G5 {15..18}, G6 {7..10}, and stored
// [group][species][direction in group], so that the planes one tile copy of
// the TMA-staged step needs (same halo shape, all species) are contiguous.
template <int LAT>
__host__ __device__ constexpr int grp(int a)
{
    return LAT == 0 ? 0
                    : (a == 0 ? 0 : (a == 5 || a == 6) ? 1 : (a == 1 || a == 2) ? 2 : (a >= 11 && a <= 14) ? 3
                       : (a == 3 || a == 4) ? 4 : (a >= 15) ? 5 : 6);
}
__host__ __device__ constexpr int grp_start(int g)
{
    return g == 0 ? 0 : g == 1 ? 1 : g == 2 ? 3 : g == 3 ? 5 : g == 4 ? 9 : g == 5 ? 11 : 15;
}
__host__ __device__ constexpr int grp_size(int g) { return g == 0 ? 1 : (g == 1 || g == 2 || g == 4) ? 2 : 4; }
template <int LAT>
__host__ __device__ constexpr int grp_pos(int a)
{
    return LAT == 0 ? a
                    : (a == 0 ? 0 : (a == 5 || a == 6) ? a - 5 : (a == 1 || a == 2) ? a - 1
                       : (a >= 11 && a <= 14) ? a - 11 : (a == 3 || a == 4) ? a - 3 : (a >= 15) ? a - 15 : a - 7);
}
template <int LAT, int NS>
__host__ __device__ constexpr int plane_of(int i, int a)
{
    return LAT == 0 ? i * 9 + a
                    : NS * grp_start(grp<LAT>(a)) + i * grp_size(grp<LAT>(a)) + grp_pos<LAT>(a);
}

// Plane of the stored node densities rho~_i of species i (half storage):
// after the NS * Q population planes.
template <int LAT, int NS>
__host__ __device__ constexpr int ref_plane(int i)
{
    return NS * Lat<LAT>::Q + i;
}

// --------------------------------------------------------------- parameters
// Per-run constants, computed on the host in double and cast to T.
template <typename T>
struct Params {
    int nx, ny, nz, nsites;
    long long pstride;
    int wall[3];           // 1 if that dimension is closed by walls at both ends
    int unit[MAXS];        // species moves exactly one node per step (c == 1)
    T c[MAXS];             // lattice speed c_i = sqrt(M_1 / M_i)
    T inv_cs2[MAXS];       // 1 / c_s,i^2 = 3 / c_i^2
    T c_inv_cs2[MAXS];     // c_i / c_s,i^2 = 3 / c_i
    T c_inv_cs2_lo[MAXS];  // float arithmetic: c_inv_cs2 + c_inv_cs2_lo = 1 / (c_i m2) (0 in double)
    T tau_inv[MAXS];       // 1 / tau_i
    T omt[MAXS];           // 1 - 1/tau_i
    T sfac[MAXS];          // 1 - 1/(2 tau_i)
    T Minv[MAXS];          // 1 / M_i
    T M[MAXS];
    T MM[MAXS][MAXS];      // 2 n^2 M_i M_j / (p dt) = n * MM_ij  (p = n M_1 / 3)
    T iD[MAXS][MAXS];      // 1 / D_ij
    T g[3];                // specific body force
    T w1[MAXS][3];         // 1-D interpolation weights: [upstream, centre, downstream]
    T w2[MAXS][3][3];      // products w1[a] * w1[b]
    T wl[3];               // lattice weight per class (rest, axis, diagonal)
    T ref[MAXS][3];        // deviation reference per class: wl[class] * rho_ref_i
    // float storage computes in deviations g = f - ref (see Codec::DARITH):
    T rref[MAXS];          // sum over directions of ref: the density g = 0 stands for
    T refc[MAXS][3];       // wl[class] * rref - ref[class], the rounding of ref, exactly
    const T* kf;           // per-node specific force [3][nsites] added to g, or nullptr
    unsigned flags;        // corrective forcing terms: bit 0 S_diff, 1 S_p, 2 S_rho
    const T* rhof;         // [ns + 1][nsites] densities of f_t (species, mixture) or nullptr
    unsigned seed;         // per-step seed of the dithered rounding of reduced storage (0: off)
};

template <typename T>
inline Params<T> to_params(const HostParams& h)
{
    Params<T> p;
    p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.nsites = h.nsites;
    p.pstride = h.pstride;
    for (int k = 0; k < 3; ++k) { p.wall[k] = h.wall[k]; p.g[k] = (T)h.g[k]; p.wl[k] = (T)h.wl[k]; }
    for (int i = 0; i < MAXS; ++i) {
        p.unit[i] = h.unit[i];
        p.c[i] = (T)h.c[i]; p.inv_cs2[i] = (T)h.inv_cs2[i]; p.c_inv_cs2[i] = (T)h.c_inv_cs2[i];
        p.c_inv_cs2_lo[i] = (T)h.c_inv_cs2_lo[i];
        p.tau_inv[i] = (T)h.tau_inv[i]; p.omt[i] = (T)h.omt[i]; p.sfac[i] = (T)h.sfac[i];
        p.Minv[i] = (T)h.Minv[i]; p.M[i] = (T)h.M[i];
        for (int j = 0; j < MAXS; ++j) { p.MM[i][j] = (T)h.MM[i][j]; p.iD[i][j] = (T)h.iD[i][j]; }
        for (int a = 0; a < 3; ++a) {
            p.w1[i][a] = (T)h.w1[i][a];
            p.ref[i][a] = (T)h.ref[i][a];
            for (int b = 0; b < 3; ++b) p.w2[i][a][b] = (T)h.w2[i][a][b];
        }
    }
    p.kf = (const T*)h.kf;
    p.flags = h.flags;
    p.rhof = (const T*)h.rhof;
    p.seed = h.seed;
    // directions per class: rest, axis, diagonal
    const double n1 = h.lattice == 0 ? 4.0 : 6.0, n2 = h.lattice == 0 ? 4.0 : 12.0;
    for (int i = 0; i < MAXS; ++i) {
        const double r0 = (double)p.ref[i][0], r1 = (double)p.ref[i][1], r2 = (double)p.ref[i][2];
        p.rref[i] = (T)(r0 + n1 * r1 + n2 * r2);
        for (int a = 0; a < 3; ++a) p.refc[i][a] = (T)((double)p.wl[a] * (double)p.rref[i] - (double)p.ref[i][a]);
    }
    return p;
}

// --------------------------------------------------------- storage codecs
// Raw double storage; float storage of the deviation f - w_a rho_ref_i from
// one reference density per species; float storage of the deviation from the
// node's own density (f32n); half storage of the deviation f - w_a rho~_i(x)
// from the node's own density rho~_i(x), which is stored (as a half, so
// exactly) in one extra plane per species.  A stored value at node X decodes
// with the reference of X itself.
//
// Flags:
//   DEV      populations are stored as deviations from a reference
//   LOCAL    the reference is per node (stored next to the deviations)
//   DARITH   the moments and the collision work on deviations from one
//            reference density per species (rref)
//   NODE     the gather, the moments and the collision work on deviations
//            from the node's own reference density: a stencil value at X
//            enters the node O as g(X) + w_a (rho~(X) - rho~(O))
//   REST_IMPLIED  the rest plane holds the node's density itself; the rest
//            deviation is minus the sum of the other deviations (the
//            deviations of a post-collision state sum to zero), so the node
//            reference costs no extra bytes
template <typename S> struct Codec;
template <> struct Codec<double> {
    static constexpr bool DEV = false;
    static constexpr bool LOCAL = false;
    static constexpr bool DARITH = false;
    static constexpr bool NODE = false;
    static constexpr bool REST_IMPLIED = false;
    static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <> struct Codec<float> {
    static constexpr bool DEV = true;
    static constexpr bool LOCAL = false;
    // arithmetic on the deviations g = f - ref themselves: the gather, the
    // moments (rho = rref + sum g, j = sum e g) and the collision never form
    // the full-size populations, whose float rounding would swamp the small
    // momenta and forcing terms of near-rest mixtures
    static constexpr bool DARITH = true;
    static constexpr bool NODE = false;
    static constexpr bool REST_IMPLIED = false;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
// Float storage element of the node-reference encoding (same bits as a float).
struct f32n {
    float v;
};
template <> struct Codec<f32n> {
    static constexpr bool DEV = true;
    static constexpr bool LOCAL = true;
    static constexpr bool DARITH = false;
    // deviations from the node's own density, which the rest plane holds: a
    // species depleted a thousandfold somewhere keeps the float precision of
    // its own density there (one reference per species would spend it on the
    // mean density)
    static constexpr bool NODE = true;
    static constexpr bool REST_IMPLIED = true;
    static __device__ __forceinline__ float ld(const f32n* p) { return __ldg(reinterpret_cast<const float*>(p)); }
    static __device__ __forceinline__ void st(f32n* p, float v) { *reinterpret_cast<float*>(p) = v; }
    static __device__ __forceinline__ float rt(float v) { return v; }
};
template <> struct Codec<__half> {
    static constexpr bool DEV = true;
    static constexpr bool LOCAL = true;
    static constexpr bool DARITH = false;
    static constexpr bool NODE = true;
    static constexpr bool REST_IMPLIED = false;
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    // the value a float takes once stored
    static __device__ __forceinline__ float rt(float v) { return __half2float(__float2half_rn(v)); }
};

// ------------------------------------------------------ dithered rounding
// A slowly varying field is rounded the same way every step, so its rounding
// error adds up like a steady source instead of averaging out; over tens of
// thousands of steps that frozen error, not the random part, decides the
// reduced-precision error.  Reduced storage therefore rounds its last
// operation with a dither: a uniform offset of up to half a unit in the last
// place of the result's precision, drawn from a counter-based hash of (seed of
// the step, node, species, direction), is added before rounding to nearest,
// which makes the rounding error zero-mean and uncorrelated from step to step.
__device__ __forceinline__ unsigned dither_hash(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Signed uniform in [-1/2, 1/2) times u, from 32 hash bits.
__device__ __forceinline__ float dither_scale(unsigned h, float u)
{
    return (float)(int)h * (u * 2.3283064365386963e-10f);
}

// One unit in the last place of v in float (0 for |v| below 2^-102).
__device__ __forceinline__ float ulp_float(float v)
{
    const int e = __float_as_int(v) & 0x7f800000;
    return e > (23 << 23) ? __int_as_float(e - (23 << 23)) : 0.0f;
}

// One unit in the last place of v once stored as a half (subnormal halves: 2^-24).
__device__ __forceinline__ float ulp_half(float v)
{
    const int e = __float_as_int(v) & 0x7f800000;
    return e >= ((127 - 14) << 23) ? __int_as_float(e - (10 << 23)) : 5.9604644775390625e-8f;
}

// Plane holding the node reference densities of species i (node encodings).
template <int LAT, int NS, typename S>
__host__ __device__ constexpr int node_ref_plane(int i)
{
    return Codec<S>::REST_IMPLIED ? plane_of<LAT, NS>(i, 0) : ref_plane<LAT, NS>(i);
}

// The densities the deviations of a node are taken from, per species: the
// node's own stored references (node encodings), the per-species references
// (DARITH), zero (raw storage).
template <int LAT, int NS, typename S, typename T>
__device__ __forceinline__ void node_base(const Params<T>& p, const S* __restrict__ fin, int node, T (&R)[NS])
{
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        if constexpr (Codec<S>::NODE)
            R[i] = (T)Codec<S>::ld(fin + (long long)node_ref_plane<LAT, NS, S>(i) * p.pstride + node);
        else if constexpr (Codec<S>::DARITH)
            R[i] = p.rref[i];
        else
            R[i] = (T)0;
    }
}

// Arithmetic on deviations (from one reference per species, or per node).
template <typename S>
__host__ __device__ constexpr bool dev_arith()
{
    return Codec<S>::DARITH || Codec<S>::NODE;
}

// ------------------------------------------------------------- neighbours
// off[k][o+1]: element offset of the node at o in {-1,0,+1} along dimension k
// (periodic wrap; 0 when that node is solid).  lo/hi: the node touches the
// low/high wall of dimension k.
struct Nbr {
    int off[3][3];
    bool lo[3], hi[3];
    bool any_wall;
};

template <typename T>
__device__ __forceinline__ Nbr neighbours(const Params<T>& p, int node)
{
    Nbr nb;
    const int nxy = p.nx * p.ny;
    const int crd[3] = {node % p.nx, (node / p.nx) % p.ny, node / nxy};
    const int stride[3] = {1, p.nx, nxy};
    const int ext[3] = {p.nx, p.ny, p.nz};
    nb.any_wall = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool at_lo = crd[k] == 0, at_hi = crd[k] == ext[k] - 1;
        nb.lo[k] = p.wall[k] && at_lo;
        nb.hi[k] = p.wall[k] && at_hi;
        nb.any_wall |= nb.lo[k] | nb.hi[k];
        nb.off[k][1] = 0;
        nb.off[k][0] = at_lo ? (p.wall[k] ? 0 : (ext[k] - 1) * stride[k]) : -stride[k];
        nb.off[k][2] = at_hi ? (p.wall[k] ? 0 : -(ext[k] - 1) * stride[k]) : stride[k];
    }
    return nb;
}

// 1-D weight index of source offset o along a dimension whose unit velocity
// component is e (!= 0): upstream (o == -e) 0, centre 1, downstream 2.
__host__ __device__ constexpr int widx(int o, int e) { return o == -e ? 0 : (o == 0 ? 1 : 2); }

// -------------------------------------------------------------- the gather
// Interior node: f_a(O) = sum over the 1/3/9 stencil nodes O + o of
// W(o) f*_a(O + o), the tensor product of 1-D weights along the (one or two)
// dimensions direction a moves in.
// Storage decodes: raw values (FP64); deviations from one reference per
// species, interpolated as they are (the weights sum to exactly one); node
// encodings: the deviation relative to O's own reference R_O,
// g(X) + w_a (R(X) - R_O), whose interpolant is the deviation of f_a(O)
// from w_a R_O (R0 = R_O).
template <int LAT, int NS, int I, int A, typename S, typename T>
__device__ __forceinline__ T gather_interior(const Params<T>& p, const S* __restrict__ fin, int node,
                                             const Nbr& nb, T R0)
{
    constexpr int ex = ev<LAT>(A, 0), ey = ev<LAT>(A, 1), ez = ev<LAT>(A, 2);
    const S* plane = fin + (long long)plane_of<LAT, NS>(I, A) * p.pstride + node;
    const S* rplane = fin + (long long)node_ref_plane<LAT, NS, S>(I) * p.pstride + node;
    const T wa = p.wl[wclass<LAT>(A)];
    // the stored value at offset o, decoded relative to O's own reference
    // where the storage keeps one per node
    auto ldv = [&](long long o) -> T {
        if constexpr (Codec<S>::NODE) return fma(wa, (T)Codec<S>::ld(rplane + o) - R0, (T)Codec<S>::ld(plane + o));
        else return (T)Codec<S>::ld(plane + o);
    };
    T acc;
    if constexpr (ex == 0 && ey == 0 && ez == 0) {
        acc = ldv(0);
    } else {
        if (p.unit[I]) {
            acc = ldv(nb.off[0][1 - ex] + nb.off[1][1 - ey] + nb.off[2][1 - ez]);
        } else {
            constexpr int k1 = ex != 0 ? 0 : (ey != 0 ? 1 : 2);
            constexpr int k2 = (ex != 0 && ey != 0) ? 1 : (((ex != 0 || ey != 0) && ez != 0) ? 2 : -1);
            constexpr int e1 = ev<LAT>(A, k1);
            acc = (T)0;
            if constexpr (k2 < 0) {
#pragma unroll
                for (int o1 = -1; o1 <= 1; ++o1)
                    acc += p.w1[I][widx(o1, e1)] * ldv(nb.off[k1][o1 + 1]);
            } else if constexpr (std::is_same<T, double>::value) {
                constexpr int e2 = ev<LAT>(A, k2);
#pragma unroll
                for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
                    for (int o1 = -1; o1 <= 1; ++o1)
                        acc += p.w2[I][widx(o1, e1)][widx(o2, e2)] * ldv(nb.off[k1][o1 + 1] + nb.off[k2][o2 + 1]);
            } else {
                // float arithmetic: two 1-D passes, so that the effective 2-D
                // weights are products of 1-D weights that sum to exactly one
                constexpr int e2 = ev<LAT>(A, k2);
#pragma unroll
                for (int o2 = -1; o2 <= 1; ++o2) {
                    T row = (T)0;
#pragma unroll
                    for (int o1 = -1; o1 <= 1; ++o1)
                        row += p.w1[I][widx(o1, e1)] * ldv(nb.off[k1][o1 + 1] + nb.off[k2][o2 + 1]);
                    acc += p.w1[I][widx(o2, e2)] * row;
                }
            }
        }
    }
    return acc;
}

// Push weight of direction B from a node X to X + d (the interpolation read as
// a redistribution of each streamed value, as App. A does).
template <int LAT, int B, typename T>
__device__ __forceinline__ T push_weight(const Params<T>& p, int I, int dx, int dy, int dz)
{
    const int d[3] = {dx, dy, dz};
    T w = (T)1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int e = ev<LAT>(B, k);
        if (e != 0) w *= p.w1[I][d[k] == e ? 0 : (d[k] == 0 ? 1 : 2)];
    }
    return w;
}

// App. A lumping at a wall-adjacent node O for direction B leaving O: weight
// bound for a solid node O + d stays at O, in the opposite direction when B
// heads into the crossed wall(s) (e_B . d_s > 0, d_s the crossing components
// of d), and in B itself otherwise (ties at edges and corners included).
// Returns the weight kept in B (into_self) or sent to the opposite of B.
template <int LAT, int B, typename T>
__device__ __forceinline__ T lumped(const Params<T>& p, int I, const Nbr& nb, bool into_self)
{
    constexpr int ex = ev<LAT>(B, 0), ey = ev<LAT>(B, 1), ez = ev<LAT>(B, 2);
    T acc = (T)0;
#pragma unroll
    for (int dz = (ez ? -1 : 0); dz <= (ez ? 1 : 0); ++dz)
#pragma unroll
        for (int dy = (ey ? -1 : 0); dy <= (ey ? 1 : 0); ++dy)
#pragma unroll
            for (int dx = (ex ? -1 : 0); dx <= (ex ? 1 : 0); ++dx) {
                const int d[3] = {dx, dy, dz};
                bool crossed = false;
                int dot = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const bool cr = (d[k] == 1 && nb.hi[k]) || (d[k] == -1 && nb.lo[k]);
                    crossed |= cr;
                    if (cr) dot += ev<LAT>(B, k) * d[k];
                }
                if (crossed && ((dot > 0) != into_self)) acc += push_weight<LAT, B>(p, I, dx, dy, dz);
            }
    return acc;
}

// Wall-adjacent node: only fluid stencil nodes contribute, plus the lumped
// weight of O's own populations in directions a and its opposite.
template <int LAT, int NS, int I, int A, typename S, typename T>
__device__ __forceinline__ T gather_wall(const Params<T>& p, const S* __restrict__ fin, int node,
                                         const Nbr& nb, T R0)
{
    constexpr int ex = ev<LAT>(A, 0), ey = ev<LAT>(A, 1), ez = ev<LAT>(A, 2);
    constexpr int AB = opp<LAT>(A);
    const S* plane = fin + (long long)plane_of<LAT, NS>(I, A) * p.pstride + node;
    const S* rplane = fin + (long long)node_ref_plane<LAT, NS, S>(I) * p.pstride + node;
    const T wa = p.wl[wclass<LAT>(A)];
    // deviation storage gathers deviations; the reference carried by the
    // weights of this node, ref * (K - 1) with K the sum of the fluid stencil
    // weights and the lumped ones, is added at the end (K = 1 away from walls)
    T ksum = (T)0;
    // stored value of plane q at offset o, decoded relative to O's reference
    // where the storage keeps one per node
    auto ldv = [&](const S* q, long long o) -> T {
        if constexpr (Codec<S>::NODE) return fma(wa, (T)Codec<S>::ld(rplane + o) - R0, (T)Codec<S>::ld(q + o));
        else return (T)Codec<S>::ld(q + o);
    };
    T acc = (T)0;
#pragma unroll
    for (int oz = (ez ? -1 : 0); oz <= (ez ? 1 : 0); ++oz)
#pragma unroll
        for (int oy = (ey ? -1 : 0); oy <= (ey ? 1 : 0); ++oy)
#pragma unroll
            for (int ox = (ex ? -1 : 0); ox <= (ex ? 1 : 0); ++ox) {
                const bool solid = (ox == -1 && nb.lo[0]) || (ox == 1 && nb.hi[0]) ||
                                   (oy == -1 && nb.lo[1]) || (oy == 1 && nb.hi[1]) ||
                                   (oz == -1 && nb.lo[2]) || (oz == 1 && nb.hi[2]);
                if (!solid) {
                    const T w = push_weight<LAT, A>(p, I, -ox, -oy, -oz);  // from O + o to O: d = -o
                    acc += w * ldv(plane, nb.off[0][ox + 1] + nb.off[1][oy + 1] + nb.off[2][oz + 1]);
                    ksum += w;
                }
            }
    if constexpr (ex != 0 || ey != 0 || ez != 0) {
        const T ls = lumped<LAT, A>(p, I, nb, true);
        const T lo = lumped<LAT, AB>(p, I, nb, false);
        if (ls != (T)0) acc += ls * ldv(plane, 0);
        if (lo != (T)0) acc += lo * ldv(fin + (long long)plane_of<LAT, NS>(I, AB) * p.pstride + node, 0);
        ksum += ls + lo;
    }
    if constexpr (Codec<S>::DARITH) acc += p.ref[I][wclass<LAT>(A)] * (ksum - (T)1);
    if constexpr (Codec<S>::NODE) acc += wa * R0 * (ksum - (T)1);
    return acc;
}

// Node encodings with the rest plane holding the density: the rest deviation
// of O is minus the sum of O's stored deviations in the other directions.
template <int LAT, int NS, int I, typename S, typename T>
__device__ __forceinline__ T implied_rest(const Params<T>& p, const S* __restrict__ fin, int node)
{
    T acc = (T)0;
    static_for<1, Lat<LAT>::Q>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        acc -= (T)Codec<S>::ld(fin + (long long)plane_of<LAT, NS>(I, A) * p.pstride + node);
    });
    return acc;
}

// f: the gathered populations (raw) or their deviations from R0 (the node's
// own references, or the per-species ones).
template <int LAT, int NS, typename S, typename T>
__device__ __forceinline__ void gather_all(const Params<T>& p, const S* __restrict__ fin, int node,
                                           const Nbr& nb, const T (&R0)[NS], T (&f)[NS][Lat<LAT>::Q])
{
    constexpr int Q = Lat<LAT>::Q;
    constexpr int A0 = Codec<S>::REST_IMPLIED ? 1 : 0;
    if constexpr (Codec<S>::REST_IMPLIED)
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            f[I][0] = implied_rest<LAT, NS, I>(p, fin, node);
        });
    if (!nb.any_wall) {
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            static_for<A0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                f[I][A] = gather_interior<LAT, NS, I, A>(p, fin, node, nb, R0[I]);
            });
        });
    } else {
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            static_for<A0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                f[I][A] = gather_wall<LAT, NS, I, A>(p, fin, node, nb, R0[I]);
            });
        });
    }
}

// Raw storage (no references): the gather of the double-precision step.
template <int LAT, int NS, typename T>
__device__ __forceinline__ void gather_all(const Params<T>& p, const double* __restrict__ fin, int node,
                                           const Nbr& nb, T (&f)[NS][Lat<LAT>::Q])
{
    const T R0[NS] = {};
    gather_all<LAT, NS>(p, fin, node, nb, R0, f);
}

// The stored state of the node itself (no streaming), decoded as the gather
// decodes: raw values, deviations from the per-species references, or
// deviations from the node's own references R0.
template <int LAT, int NS, typename S, typename T>
__device__ __forceinline__ void load_raw(const Params<T>& p, const S* __restrict__ fin, int node,
                                         T (&f)[NS][Lat<LAT>::Q])
{
    constexpr int Q = Lat<LAT>::Q;
    static_for<0, NS>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            if constexpr (Codec<S>::REST_IMPLIED && A == 0)
                f[I][0] = implied_rest<LAT, NS, I>(p, fin, node);
            else
                f[I][A] = (T)Codec<S>::ld(fin + (long long)plane_of<LAT, NS>(I, A) * p.pstride + node);
        });
    });
}

// Store the post-collision state f (raw, or deviations from R0).  rho: the
// node's species densities.  Node encodings store the new reference
// R* = rho (rounded as stored: half storage keeps it as a half) and the
// deviations from it, g - w_a (R* - R0) (R* - R0 is exact: both are close).
// DITHER (half storage, p.seed != 0): the conversion to half is dithered.
template <int LAT, int NS, typename S, bool DITHER = false, typename T>
__device__ __forceinline__ void store_all(const Params<T>& p, S* __restrict__ fout, int node,
                                          const T (&f)[NS][Lat<LAT>::Q], const T (&rho)[NS], const T (&R0)[NS],
                                          unsigned h0 = 0)
{
    constexpr int Q = Lat<LAT>::Q;
    static_for<0, NS>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        [[maybe_unused]] T dR = (T)0;
        if constexpr (Codec<S>::NODE) {
            const T rr = (T)Codec<S>::rt((float)rho[I]);
            dR = rr - R0[I];
            Codec<S>::st(fout + (long long)node_ref_plane<LAT, NS, S>(I) * p.pstride + node, (float)rr);
        }
        static_for<Codec<S>::REST_IMPLIED ? 1 : 0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            T v = f[I][A];
            if constexpr (Codec<S>::NODE) v -= p.wl[wclass<LAT>(A)] * dR;
            if constexpr (DITHER && std::is_same<S, __half>::value) {
                if (p.seed) {
                    const unsigned r = dither_hash(h0 ^ ((unsigned)(I * 32 + A) * 0x9E3779B1u));
                    v += dither_scale(r, ulp_half((float)v));
                }
            }
            Codec<S>::st(fout + (long long)plane_of<LAT, NS>(I, A) * p.pstride + node, v);
        });
    });
}

// e_a . v with the unit vector of direction A (compile-time signs)
template <int LAT, int A, typename T>
__device__ __forceinline__ T edot(const T (&v)[3])
{
    // starts from the first non-zero term: without fast-math the compiler has
    // to keep an explicit 0 + x (it differs from x in the sign of a zero), one
    // wasted add per call
    constexpr int e0 = ev<LAT>(A, 0), e1 = ev<LAT>(A, 1), e2 = ev<LAT>(A, 2);
    if constexpr (e0 != 0) {
        T s = e0 > 0 ? v[0] : -v[0];
        if constexpr (e1 == 1) s += v[1];
        if constexpr (e1 == -1) s -= v[1];
        if constexpr (e2 == 1) s += v[2];
        if constexpr (e2 == -1) s -= v[2];
        return s;
    } else if constexpr (e1 != 0) {
        T s = e1 > 0 ? v[1] : -v[1];
        if constexpr (e2 == 1) s += v[2];
        if constexpr (e2 == -1) s -= v[2];
        return s;
    } else if constexpr (e2 != 0) {
        return e2 > 0 ? v[2] : -v[2];
    } else {
        return (T)0;
    }
}

// -------------------------------------------------- moments and relaxation
// Specific body force at a node: the uniform g plus the node's entry of the
// force field when one is set (F_i = rho_i (g + k(x)); Case II of Sec. 4.2
// is such a field).
template <typename T>
__device__ __forceinline__ void node_force(const Params<T>& p, int node, T (&g)[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = p.kf ? p.g[k] + p.kf[(long long)k * p.nsites + node] : p.g[k];
}

template <int NS, typename T>
struct NodeState {
    T rho[NS];
    T ueq[NS][3];
    T u[3];
    T V[NS][3];   // sum_j (rho_j / rho) (u_i^eq - u_j^eq) / tau_ij = Theta_i / rho_i
    T drho[NS];   // sum_a g_a: rho_i - rref_i (deviation arithmetic)
    T rho_mix, n;
};

// Cross relaxation rates X_ij = 1/tau_ij of N > 3 species, the system of
// Eq. (relation_tauij_diff_coeff) that the paper solves iteratively in a
// multicomponent mixture: one equation per pair i < j (species ordered by
// molar mass),
//   A_ij X_ij + (1/D_ij) sum_{s != i,j} rho_s X_sj = B_ij,
//   A_ij = (rho_i + rho_j)/D_ij + 2 n^2 M_i M_j/(p dt),  B_ij = 2 rho/(D_ij dt),
// solved directly by Gaussian elimination with partial pivoting (NP = N(N-1)/2
// unknowns, the pairs in the order (0,1), (0,2), ..., (1,2), ...).  For N = 2
// and 3 the same system has the closed forms used above.
template <int NS, typename T>
__device__ __forceinline__ int pair_slot(int a, int b)
{
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * NS - lo * (lo + 1) / 2 + (hi - lo - 1);
}

template <int NS, typename T>
__device__ void tau_dense(const Params<T>& p, const T (&rho)[NS], T rho_mix, T n, T (&X)[MAXS][MAXS],
                          unsigned& err)
{
    constexpr int NP = NS * (NS - 1) / 2;
    T A[NP][NP + 1];
#pragma unroll
    for (int r = 0; r < NP; ++r)
#pragma unroll
        for (int c = 0; c <= NP; ++c) A[r][c] = (T)0;
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int j = i + 1; j < NS; ++j) {
            const int r = pair_slot<NS, T>(i, j);
            A[r][r] += (rho[i] + rho[j]) * p.iD[i][j] + n * p.MM[i][j];   // MM = 2 n M_i M_j/(p dt) / n
#pragma unroll
            for (int q = 0; q < NS; ++q)
                if (q != i && q != j) A[r][pair_slot<NS, T>(q, j)] += rho[q] * p.iD[i][j];
            A[r][NP] = (T)2 * rho_mix * p.iD[i][j];
        }
    for (int c = 0; c < NP; ++c) {
        int piv = c;
        for (int r = c + 1; r < NP; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(A[piv][c] != (T)0)) { err |= ERR_TAU; return; }
        if (piv != c)
            for (int k = 0; k <= NP; ++k) { const T t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        for (int r = c + 1; r < NP; ++r) {
            const T m = A[r][c] / A[c][c];
            for (int k = c; k <= NP; ++k) A[r][k] -= m * A[c][k];
        }
    }
    for (int c = NP - 1; c >= 0; --c) {
        T acc = A[c][NP];
        for (int k = c + 1; k < NP; ++k) acc -= A[c][k] * A[k][NP];
        A[c][NP] = acc / A[c][c];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int j = i + 1; j < NS; ++j) X[i][j] = X[j][i] = A[pair_slot<NS, T>(i, j)][NP];
}

// Moments (Eq. zeroth_order_moment, first_order_moment_force with F_i =
// rho_i g, Eq. Sirovich_mixture_density and _velocity), n = sum rho_i/M_i and
// the cross relaxation rates 1/tau_ij of Eq. (relation_tauij_diff_coeff):
// Eq. (Luo&Girimaji_tau) for two species and the Sec. 4.1 closed forms for
// three, written for 1/tau_ij.
// DA: f holds deviations g = f - w R0 (deviation storage): rho_i = R0_i +
// sum g, j_i = sum e g (the references cancel in j); R0 is the per-species
// reference or the node's own (node_base).
// DITHER (node references in float, p.seed != 0): rho_i = R0_i + sum g is
// rounded with a dither (h0: the node's hash of the step seed).  The node's
// density is stored as this float, and a change below half a unit in its
// last place would otherwise be lost at the same node every step.
template <int LAT, int NS, bool DA = false, bool DITHER = false, typename T>
__device__ __forceinline__ void moments(const Params<T>& p, const T (&f)[NS][Lat<LAT>::Q],
                                        NodeState<NS, T>& s, unsigned& err, const T (&g)[3],
                                        const T* R0 = nullptr, unsigned h0 = 0)
{
    constexpr int Q = Lat<LAT>::Q;
    s.rho_mix = (T)0;
    s.n = (T)0;
    static_for<0, NS>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        T r = (T)0, j[3] = {(T)0, (T)0, (T)0};
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            const T v = f[I][A];
            r += v;
            if constexpr (ev<LAT>(A, 0) == 1) j[0] += v;
            if constexpr (ev<LAT>(A, 0) == -1) j[0] -= v;
            if constexpr (ev<LAT>(A, 1) == 1) j[1] += v;
            if constexpr (ev<LAT>(A, 1) == -1) j[1] -= v;
            if constexpr (ev<LAT>(A, 2) == 1) j[2] += v;
            if constexpr (ev<LAT>(A, 2) == -1) j[2] -= v;
        });
        s.drho[I] = r;
        if constexpr (DA && DITHER) {
            if (p.seed) r += (T)dither_scale(dither_hash(h0 ^ (0x5bd1e995u * (unsigned)(I + 1))), ulp_float((float)R0[I]));
        }
        if constexpr (DA) r = R0[I] + r;
        if (!(r > (T)0)) err |= ERR_RHO;
        const T rinv = (T)1 / r;
        s.rho[I] = r;
#pragma unroll
        for (int k = 0; k < 3; ++k) s.ueq[I][k] = p.c[I] * j[k] * rinv + (T)0.5 * g[k];
        s.rho_mix += r;
        s.n += r * p.Minv[I];
    });
    const T rinv_m = (T)1 / s.rho_mix;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T acc = (T)0;
#pragma unroll
        for (int i = 0; i < NS; ++i) acc += s.rho[i] * s.ueq[i][k];
        s.u[k] = acc * rinv_m;
    }
    // X_ij = 1/tau_ij
    T X[MAXS][MAXS] = {};
    if constexpr (NS == 2) {
        const T A12 = (s.rho[0] + s.rho[1]) * p.iD[0][1] + s.n * p.MM[0][1];
        const T B12 = (T)2 * s.rho_mix * p.iD[0][1];
        X[0][1] = X[1][0] = B12 / A12;
    } else if constexpr (NS == 3) {
        const T r1 = s.rho[0], r2 = s.rho[1], r3 = s.rho[2];
        const T A12 = (r1 + r2) * p.iD[0][1] + s.n * p.MM[0][1];
        const T A13 = (r1 + r3) * p.iD[0][2] + s.n * p.MM[0][2];
        const T A23 = (r2 + r3) * p.iD[1][2] + s.n * p.MM[1][2];
        const T B12 = (T)2 * s.rho_mix * p.iD[0][1];
        const T B13 = (T)2 * s.rho_mix * p.iD[0][2];
        const T B23 = (T)2 * s.rho_mix * p.iD[1][2];
        const T rA13 = (T)1 / A13;
        const T X23 = (B23 - r1 * B13 * rA13 * p.iD[1][2]) /
                      (A23 - r1 * r2 * rA13 * p.iD[0][2] * p.iD[1][2]);
        const T X12 = (B12 - r3 * X23 * p.iD[0][1]) / A12;
        const T X13 = (B13 - r2 * X23 * p.iD[0][2]) * rA13;
        X[0][1] = X[1][0] = X12;
        X[0][2] = X[2][0] = X13;
        X[1][2] = X[2][1] = X23;
    }
    else if constexpr (NS > 3) {
        tau_dense<NS>(p, s.rho, s.rho_mix, s.n, X, err);
    }
    // tau_ij < 1/2 is a legitimate outcome of the relation (it happens for
    // trace species); only a non-positive or non-finite tau_ij is an error.
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int j = i + 1; j < NS; ++j)
            if (!(X[i][j] > (T)0) || !isfinite(X[i][j])) err |= ERR_TAU;
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T acc = (T)0;
#pragma unroll
            for (int j = 0; j < NS; ++j)
                if (j != i) acc += s.rho[j] * X[i][j] * (s.ueq[i][k] - s.ueq[j][k]);
            s.V[i][k] = acc * rinv_m;
        }
}

// Collision of Eq. (LBE_forcing) in place, f <- f*:
//   f* = f - (f - f^(0))/tau_i + sum_j Omega^ij + (1 - 1/(2 tau_i)) S
// with f^(0) = [1 + (e-u).(u_i^eq-u)/c_s^2] f^eq (Eq. feqi0),
//      sum_j Omega^ij = -(f^eq/c_s^2)(e-u).V_i (Eq. Cross_collision_Sirovich),
//      S = w [e/c_s^2 + (ee - c_s^2 I).u/c_s^4].F_i (Eq. CE_forcing_term_discretized),
// rearranged to  f* = (1 - 1/tau) f + f^eq [1/tau + (e-u).a/c_s^2] + (1-1/(2tau)) S,
//                a  = (u_i^eq - u)/tau - V_i.
// DA: f holds deviations g = f - ref and receives g* = f* - ref, written so
// that only the last addition is at the size of g:
//   g* = g + (w drho + refc - g)/tau + w rho (phi B + b) + (1 - 1/(2 tau)) S
// (1 - 1/tau = omt exactly on the float grid of the constants); refc, the
// rounding of the per-species reference, is zero for a node reference
// (NODE: ref = w R0 exactly, so w rho - ref = w drho).
// with feq = w rho (1 + phi), phi = t1 (1 + t1/2) - u^2/(2 c_s^2),
//      B = 1/tau + b, b = (e-u).a / c_s^2 (the same algebra as above, minus ref).
// CORR: add the corrective terms of Eq. (improved_forcing_scheme) that
// p.flags selects (they are part of S, so the update scales them by
// 1 - 1/(2 tau_i)): with e = c_i e_hat,
//   S_diff = w [(e e - cs2 I)/cs2^2 . u] . Theta_i dt/(2 tau_i - dt),
//   S_p    = w [(e e - cs2 I)/cs2^2 . u] . grad(rho_i cs2)      (subtracted),
//   S_rho  = w [(e e - cs2 I)/cs2 . u_i^eq] . (w_i grad rho),   w_i = rho_i/rho;
// grad: [NS + 1][3] lattice gradients of rho_i and rho at this node.
// shift (DA, node references): per species, the new reference minus the old
// one; the update then yields the deviation from the new reference in its
// one final rounding.  DITHER (float storage, p.seed != 0): that rounding is
// dithered (h0: the node's hash of the step seed).
template <int LAT, int NS, bool DA = false, bool CORR = false, bool NODE = false, bool DITHER = false, typename T>
__device__ __forceinline__ void collide(const Params<T>& p, T (&f)[NS][Lat<LAT>::Q],
                                        const NodeState<NS, T>& s, const T (&g)[3],
                                        const T (*grad)[3] = nullptr, const T* shift = nullptr,
                                        unsigned h0 = 0)
{
    constexpr int Q = Lat<LAT>::Q;
    // k x for k = c_i / c_s,i^2 (with its low part in float arithmetic, so
    // that the equilibrium carries exactly the species momentum)
    auto kmul = [&](int i, T x) -> T {
        if constexpr (std::is_same<T, float>::value) return fmaf(p.c_inv_cs2[i], x, p.c_inv_cs2_lo[i] * x);
        else return p.c_inv_cs2[i] * x;
    };
    // f <- f + X (deviation arithmetic): minus the reference shift, plus the
    // dither, in the single rounding of the last addition
    auto upd = [&](int i, int a, int c, T X) -> T {
        if (shift) X -= p.wl[c] * shift[i];
        if constexpr (DITHER) {
            if (p.seed) {
                const unsigned r = dither_hash(h0 ^ ((unsigned)(i * 32 + a) * 0x9E3779B1u));
                X += (T)dither_scale(r, ulp_float((float)(f[i][a] + X)));
            }
        }
        return f[i][a] + X;
    };
    T Xc[NS][3], Yc[NS][3];   // the vectors the corrective terms contract with
    if constexpr (CORR) {
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const T tau_i = (T)1 / p.tau_inv[i];
            const T cs2 = (T)1 / p.inv_cs2[i];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Xc[i][k] = (p.flags & 1u) ? s.rho[i] * s.V[i][k] / ((T)2 * tau_i - (T)1) : (T)0;   // Theta_i = rho_i V_i
                if (p.flags & 2u) Xc[i][k] -= cs2 * grad[i][k];
                Yc[i][k] = (p.flags & 4u) ? s.rho[i] / s.rho_mix * grad[NS][k] : (T)0;
            }
        }
    }
    const T usq = s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2];
    const T ug = s.u[0] * g[0] + s.u[1] * g[1] + s.u[2] * g[2];
    T av[NS][3], Bc[NS], U2[NS], wr[NS][3], sr[NS], Bm[NS], dt[NS][3];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        T ua = (T)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            av[i][k] = (s.ueq[i][k] - s.u[k]) * p.tau_inv[i] - s.V[i][k];
            ua += s.u[k] * av[i][k];
        }
        Bc[i] = p.tau_inv[i] - p.inv_cs2[i] * ua;
        Bm[i] = -p.inv_cs2[i] * ua;
        U2[i] = DA ? -(T)0.5 * p.inv_cs2[i] * usq : (T)1 - (T)0.5 * p.inv_cs2[i] * usq;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            wr[i][c] = p.wl[c] * s.rho[i];
            if constexpr (DA && NODE) dt[i][c] = p.wl[c] * s.drho[i];                   // w rho - ref
            else if constexpr (DA) dt[i][c] = fma(p.wl[c], s.drho[i], p.refc[i][c]);
        }
        sr[i] = s.rho[i] * p.inv_cs2[i] * p.sfac[i];
    }
    // the rest direction (and any direction that is its own opposite), as
    // written in the update above
    auto single = [&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int C = wclass<LAT>(A);
        const T eu = edot<LAT, A>(s.u);
        const T eg = edot<LAT, A>(g);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const T ea = edot<LAT, A>(av[i]);
            const T t1 = kmul(i, eu);                               // e.u / c_s^2
            T S = p.wl[C] * sr[i] * fma(p.c[i] * eg, (T)1 + t1, -ug);
            if constexpr (CORR) {
                const T eX = edot<LAT, A>(Xc[i]), eY = edot<LAT, A>(Yc[i]);
                const T uX = s.u[0] * Xc[i][0] + s.u[1] * Xc[i][1] + s.u[2] * Xc[i][2];
                const T qY = s.ueq[i][0] * Yc[i][0] + s.ueq[i][1] * Yc[i][1] + s.ueq[i][2] * Yc[i][2];
                const T eq = edot<LAT, A>(s.ueq[i]);
                const T c2 = p.c[i] * p.c[i];
                // ((e.u)(e.X) - cs2 u.X)/cs2^2 + ((e.u^eq)(e.Y) - cs2 u^eq.Y)/cs2, e = c e_hat
                const T corr = p.inv_cs2[i] * (p.inv_cs2[i] * c2 * eu * eX - uX) + (p.inv_cs2[i] * c2 * eq * eY - qY);
                S += p.wl[C] * p.sfac[i] * corr;
            }
            if constexpr (DA) {
                const T phi = fma(t1, fma((T)0.5, t1, (T)1), U2[i]);
                const T b = kmul(i, ea) + Bm[i];
                const T B = p.tau_inv[i] + b;
                f[i][A] = upd(i, A, C, fma(p.tau_inv[i], dt[i][C] - f[i][A], fma(wr[i][C], fma(phi, B, b), S)));
            } else {
                const T feq = wr[i][C] * fma(t1, fma((T)0.5, t1, (T)1), U2[i]);
                const T B = fma(p.c_inv_cs2[i], ea, Bc[i]);
                f[i][A] = fma(p.omt[i], f[i][A], fma(feq, B, S));
            }
        }
    };
    // Other directions in opposite pairs (A, -A): t1 = c e.u/c_s^2, e.a and
    // e.g change sign with e (the corrective terms do not), so each update is
    // f + (even part) +- (odd part), the parts formed once per pair:
    //   phi B = (phi_E + t1)(B_E + b_O),  phi_E = t1^2/2 + U2, b_O = c/cs2 e.a,
    //   S = K (c e.g t1 - u.g) + K c e.g,  K = w sr.
    static_for<0, Q>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int AB = opp<LAT>(A);
        if constexpr (A == AB) {
            single(ac);
        } else if constexpr (A < AB) {
            constexpr int C = wclass<LAT>(A);
            const T eu = edot<LAT, A>(s.u);
            const T eg = edot<LAT, A>(g);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const T t1 = kmul(i, eu);
                const T bO = kmul(i, edot<LAT, A>(av[i]));
                const T ceg = p.c[i] * eg;
                const T phiE = fma((T)0.5 * t1, t1, U2[i]);
                const T K = p.wl[C] * sr[i];
                T SE = K * fma(ceg, t1, -ug);
                const T SO = K * ceg;
                if constexpr (CORR) {
                    const T eX = edot<LAT, A>(Xc[i]), eY = edot<LAT, A>(Yc[i]);
                    const T uX = s.u[0] * Xc[i][0] + s.u[1] * Xc[i][1] + s.u[2] * Xc[i][2];
                    const T qY = s.ueq[i][0] * Yc[i][0] + s.ueq[i][1] * Yc[i][1] + s.ueq[i][2] * Yc[i][2];
                    const T eq = edot<LAT, A>(s.ueq[i]);
                    const T c2 = p.c[i] * p.c[i];
                    const T corr = p.inv_cs2[i] * (p.inv_cs2[i] * c2 * eu * eX - uX) + (p.inv_cs2[i] * c2 * eq * eY - qY);
                    SE += p.wl[C] * p.sfac[i] * corr;
                }
                if constexpr (DA) {   // X = phi (1/tau + b) + b, b = b_O + Bm
                    const T tB = p.tau_inv[i] + Bm[i];
                    const T E = fma(wr[i][C], fma(phiE, tB, fma(t1, bO, Bm[i])), SE);
                    const T O = fma(wr[i][C], fma(t1, tB, fma(phiE, bO, bO)), SO);
                    f[i][A] = upd(i, A, C, fma(p.tau_inv[i], dt[i][C] - f[i][A], E + O));
                    f[i][AB] = upd(i, AB, C, fma(p.tau_inv[i], dt[i][C] - f[i][AB], E - O));
                } else {              // B = b_O + Bc
                    const T E = fma(wr[i][C], fma(phiE, Bc[i], t1 * bO), SE);
                    const T O = fma(wr[i][C], fma(t1, Bc[i], phiE * bO), SO);
                    f[i][A] = fma(p.omt[i], f[i][A], E + O);
                    f[i][AB] = fma(p.omt[i], f[i][AB], E - O);
                }
            }
        }
    });
}

// ------------------------------------------------------ block reductions
// Per-block partial of sum rho_i in double; a fixed-order second pass
// (mass_finish) makes the total reproducible.
template <int NS, typename T>
__device__ __forceinline__ void block_mass(const T (&rho)[NS], bool active, double* __restrict__ part)
{
    __shared__ double sm[NS][BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        double v = active ? (double)rho[i] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sm[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < BLOCK / 32; ++w) t += sm[threadIdx.x][w];
        part[(long long)blockIdx.x * NS + threadIdx.x] = t;
    }
}

// ----------------------------------------------------------------- kernels
// One time step: gather f*_{t-1} -> f_t, collide -> f*_t.
// Re-injection of a species-mass deficit in proportion to the local density:
// corr_i = (m0_i - m_i) / m_i (the FP64 totals), and every node adds
// corr_i rho_i(x) to its density as f_a += w_a corr_i rho_i(x), which keeps
// the moments' shape.  A trace species thus receives (or loses) mass where it
// is abundant, in proportion to what its rounding can have lost there,
// instead of the same amount at every node.  R0: the references the
// deviations f are taken from (rho_i = R0_i + sum_a f_a).
template <int LAT, int NS, typename T>
__device__ __forceinline__ void add_correction(const Params<T>& p, const double* __restrict__ corr,
                                               T (&f)[NS][Lat<LAT>::Q], const T (&R0)[NS])
{
    static_for<0, NS>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        T r = R0[I];
        static_for<0, Lat<LAT>::Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            r += f[I][A];
        });
        const T ci = (T)__ldg(corr + I) * r;
        static_for<0, Lat<LAT>::Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            f[I][A] = fma(p.wl[wclass<LAT>(A)], ci, f[I][A]);
        });
    });
}

// The whole step at one node (gather, correction, moments, collision, store);
// s receives the node's moments (its densities feed the mass partials).
template <int LAT, int NS, typename S, typename T>
__device__ __forceinline__ void step_node(const Params<T>& p, const S* __restrict__ fin, S* __restrict__ fout,
                                          int node, const double* __restrict__ corr, NodeState<NS, T>& s,
                                          unsigned& err)
{
    constexpr int Q = Lat<LAT>::Q;
    constexpr bool DA = dev_arith<S>();
    T f[NS][Q];
    T gn[3];   // specific body force at this node
    node_force(p, node, gn);
    const Nbr nb = neighbours(p, node);
    T R0[NS];
    node_base<LAT, NS>(p, fin, node, R0);
    gather_all<LAT, NS>(p, fin, node, nb, R0, f);
    if (corr) add_correction<LAT, NS>(p, corr, f, R0);
    constexpr bool FLT = !std::is_same<S, double>::value && !std::is_same<S, __half>::value;
    constexpr bool HLF = std::is_same<S, __half>::value;
    const unsigned h0 = dither_hash(p.seed ^ ((unsigned)node * 0x85EBCA77u));
    moments<LAT, NS, DA, Codec<S>::NODE && FLT>(p, f, s, err, gn, R0, h0);
    if constexpr (Codec<S>::NODE && FLT) {
        // node references: the collision yields the deviation from the new
        // reference rho_i (the shift from the old one folded into its last
        // rounding), which store_all then keeps as is
        T Rn[NS], sh[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) { Rn[i] = (T)Codec<S>::rt((float)s.rho[i]); sh[i] = Rn[i] - R0[i]; }
        collide<LAT, NS, DA, false, true, true>(p, f, s, gn, (const T(*)[3])nullptr, sh, h0);
        store_all<LAT, NS, S>(p, fout, node, f, s.rho, Rn);
    } else {
        collide<LAT, NS, DA, false, Codec<S>::NODE, FLT>(p, f, s, gn, (const T(*)[3])nullptr, (const T*)nullptr, h0);
        store_all<LAT, NS, S, HLF>(p, fout, node, f, s.rho, R0, h0);
    }
}

template <int LAT, int NS, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_step(const Params<T> p, const S* __restrict__ fin, S* __restrict__ fout,
       double* __restrict__ mass_part, unsigned* __restrict__ err_flag, int flags,
       const double* __restrict__ corr)
{
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    const bool active = node < p.nsites;
    NodeState<NS, T> s;
    unsigned err = 0;
    if (active) {
        step_node<LAT, NS>(p, fin, fout, node, corr, s, err);
        if (err) atomicOr(err_flag, err);
    }
    if (flags & F_MASS) block_mass<NS>(s.rho, active, mass_part);
}

// Densities of f_t at every node (the gather and correction of k_step, then
// rho_i and rho), for the gradients of the corrective terms: rhof [NS + 1][nsites].
template <int LAT, int NS, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_density(const Params<T> p, const S* __restrict__ fin, T* __restrict__ rhof, const double* __restrict__ corr)
{
    constexpr int Q = Lat<LAT>::Q;
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    if (node >= p.nsites) return;
    T f[NS][Q];
    const Nbr nb = neighbours(p, node);
    T R0[NS];
    node_base<LAT, NS>(p, fin, node, R0);
    gather_all<LAT, NS>(p, fin, node, nb, R0, f);
    if (corr) add_correction<LAT, NS>(p, corr, f, R0);
    T mix = (T)0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        T r = (T)0;
#pragma unroll
        for (int a = 0; a < Q; ++a) r += f[i][a];
        if constexpr (dev_arith<S>()) r = R0[i] + r;
        rhof[(long long)i * p.nsites + node] = r;
        mix += r;
    }
    rhof[(long long)NS * p.nsites + node] = mix;
}

// Isotropic lattice gradient (1/cs0^2) sum_a w_a e_a phi(node + e_a) of a
// node field (cs0^2 = 1/3); a neighbour beyond a wall (in any component)
// takes the node's own value, periodic faces wrap.
template <int LAT, typename T>
__device__ __forceinline__ void lattice_grad(const Params<T>& p, const Nbr& nb, const T* __restrict__ phi, int node,
                                             T (&gr)[3])
{
    const T own = phi[node];
    gr[0] = gr[1] = gr[2] = (T)0;
    static_for<1, Lat<LAT>::Q>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int ex = ev<LAT>(A, 0), ey = ev<LAT>(A, 1), ez = ev<LAT>(A, 2);
        const bool solid = (ex == -1 && nb.lo[0]) || (ex == 1 && nb.hi[0]) || (ey == -1 && nb.lo[1]) ||
                           (ey == 1 && nb.hi[1]) || (ez == -1 && nb.lo[2]) || (ez == 1 && nb.hi[2]);
        const T v = solid ? own : phi[node + nb.off[0][ex + 1] + nb.off[1][ey + 1] + nb.off[2][ez + 1]];
        const T wv = p.wl[wclass<LAT>(A)] * v;
        if constexpr (ex != 0) gr[0] += ex * wv;
        if constexpr (ey != 0) gr[1] += ey * wv;
        if constexpr (ez != 0) gr[2] += ez * wv;
    });
#pragma unroll
    for (int k = 0; k < 3; ++k) gr[k] *= (T)3;
}

// The step with the corrective forcing terms p.flags selects (k_step plus
// the gradients of the densities k_density wrote for f_t).
template <int LAT, int NS, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_step_corr(const Params<T> p, const S* __restrict__ fin, S* __restrict__ fout,
            double* __restrict__ mass_part, unsigned* __restrict__ err_flag, int flags,
            const double* __restrict__ corr)
{
    constexpr int Q = Lat<LAT>::Q;
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    const bool active = node < p.nsites;
    T f[NS][Q];
    T gn[3] = {p.g[0], p.g[1], p.g[2]};
    if (active) node_force(p, node, gn);
    NodeState<NS, T> s;
    unsigned err = 0;
    if (active) {
        const Nbr nb = neighbours(p, node);
        T R0[NS];
        node_base<LAT, NS>(p, fin, node, R0);
        gather_all<LAT, NS>(p, fin, node, nb, R0, f);
        if (corr) add_correction<LAT, NS>(p, corr, f, R0);
        moments<LAT, NS, dev_arith<S>()>(p, f, s, err, gn, R0);
        T grad[NS + 1][3] = {};
        if (p.rhof)   // only the gradient terms (S_p, S_rho) have a density field
#pragma unroll
            for (int i = 0; i <= NS; ++i) lattice_grad<LAT>(p, nb, p.rhof + (long long)i * p.nsites, node, grad[i]);
        collide<LAT, NS, dev_arith<S>(), true, Codec<S>::NODE>(p, f, s, gn, grad);
        store_all<LAT, NS>(p, fout, node, f, s.rho, R0);
        if (err) atomicOr(err_flag, err);
    }
    if (flags & F_MASS) block_mass<NS>(s.rho, active, mass_part);
}

// Observables of f_t: gathered from f*_{t-1}, or read directly when the
// buffer holds f_t itself (F_RAW, right after initialisation).
template <int LAT, int NS, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_readout(const Params<T> p, const S* __restrict__ fin, int flags, double* __restrict__ x,
          double* __restrict__ rho, double* __restrict__ u, double* __restrict__ ui,
          double* __restrict__ fpop, double* __restrict__ mass_part, unsigned* __restrict__ err_flag,
          const double* __restrict__ corr)
{
    constexpr int Q = Lat<LAT>::Q, D = Lat<LAT>::D;
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    const bool active = node < p.nsites;
    T f[NS][Q];
    T gn[3] = {p.g[0], p.g[1], p.g[2]};   // specific body force at this node
    if (active) node_force(p, node, gn);
    NodeState<NS, T> s;
    unsigned err = 0;
    if (active) {
        T R0[NS];
        node_base<LAT, NS>(p, fin, node, R0);
        if (flags & F_RAW) {
            load_raw<LAT, NS>(p, fin, node, f);
        } else {
            const Nbr nb = neighbours(p, node);
            gather_all<LAT, NS>(p, fin, node, nb, R0, f);
            if (corr) add_correction<LAT, NS>(p, corr, f, R0);   // as the last step saw f_t
        }
        moments<LAT, NS, dev_arith<S>()>(p, f, s, err, gn, R0);
        const long long ns_ = p.nsites;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            if (x) x[i * ns_ + node] = (double)(s.rho[i] * p.Minv[i]) / (double)s.n;
            if (rho) rho[i * ns_ + node] = (double)s.rho[i];
#pragma unroll
            for (int k = 0; k < D; ++k)   // u_i = u_i^eq - Theta_i/(2 rho_i), Eq. (CE_EQ83)
                if (ui) ui[(i * D + k) * ns_ + node] = (double)(s.ueq[i][k] - (T)0.5 * s.V[i][k]);
        }
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (u) u[k * ns_ + node] = (double)s.u[k];
        if (fpop) {
#pragma unroll
            for (int i = 0; i < NS; ++i)
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    double v = (double)f[i][a];
                    if constexpr (Codec<S>::DARITH) v += (double)p.ref[i][wclass<LAT>(a)];
                    if constexpr (Codec<S>::NODE) v += (double)p.wl[wclass<LAT>(a)] * (double)R0[i];
                    fpop[(i * Q + a) * ns_ + node] = v;
                }
        }
        if (err) atomicOr(err_flag, err);
    }
    block_mass<NS>(s.rho, active, mass_part);
}

// Decode of a node-reference float buffer into full-size doubles (layout as
// double storage, the same plane stride).
template <int LAT, int NS>
__global__ void __launch_bounds__(BLOCK)
k_decode_f32n(const Params<float> p, const f32n* __restrict__ fin, double* __restrict__ fout)
{
    constexpr int Q = Lat<LAT>::Q;
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    if (node >= p.nsites) return;
    float R0[NS], f[NS][Q];
    node_base<LAT, NS>(p, fin, node, R0);
    load_raw<LAT, NS>(p, fin, node, f);
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
        for (int a = 0; a < Q; ++a)
            fout[(long long)plane_of<LAT, NS>(i, a) * p.pstride + node] =
                (double)p.wl[wclass<LAT>(a)] * (double)R0[i] + (double)f[i][a];
}

// Full-size populations of a node (the initial state) into the arithmetic of
// the storage: R0 receives the references (the node's own densities for the
// node encodings, rounded as stored; the per-species references for DARITH;
// zero for raw storage) and f the deviations from them.
template <int LAT, int NS, typename S, typename T>
__device__ __forceinline__ void to_deviations(const Params<T>& p, T (&f)[NS][Lat<LAT>::Q], T (&R0)[NS])
{
    constexpr int Q = Lat<LAT>::Q;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        if constexpr (Codec<S>::NODE) {
            T r = (T)0;
#pragma unroll
            for (int a = 0; a < Q; ++a) r += f[i][a];
            R0[i] = (T)Codec<S>::rt((float)r);
        } else if constexpr (Codec<S>::DARITH) {
            R0[i] = p.rref[i];
        } else {
            R0[i] = (T)0;
        }
    }
    if constexpr (dev_arith<S>())
        static_for<0, NS>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            static_for<0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                if constexpr (Codec<S>::NODE) f[I][A] -= p.wl[wclass<LAT>(A)] * R0[I];
                else f[I][A] -= p.ref[I][wclass<LAT>(A)];
            });
        });
}

// Initial state f_0 into fprev (kept for the time-0 readout) and its collision
// f*_0 into fcur.  f_0 comes from mole fractions x and number density n
// (rho_i = x_i M_i n, f = w rho_i [1 + e.u_i0 / c_s^2], u_i0 = -g/2), or from
// caller populations fsrc [ns][Q][nsites] when fsrc != nullptr.
template <int LAT, int NS, typename S, typename T>
__global__ void __launch_bounds__(BLOCK)
k_init(const Params<T> p, const double* __restrict__ xf, const double* __restrict__ nf,
       const double* __restrict__ fsrc, S* __restrict__ fprev, S* __restrict__ fcur,
       double* __restrict__ mass_part, unsigned* __restrict__ err_flag)
{
    constexpr int Q = Lat<LAT>::Q;
    const int node = blockIdx.x * BLOCK + threadIdx.x;
    const bool active = node < p.nsites;
    T f[NS][Q];
    T gn[3] = {p.g[0], p.g[1], p.g[2]};   // specific body force at this node
    if (active) node_force(p, node, gn);
    NodeState<NS, T> s;
    unsigned err = 0;
    if (active) {
        const long long ns_ = p.nsites;
        if (fsrc) {
#pragma unroll
            for (int i = 0; i < NS; ++i)
#pragma unroll
                for (int a = 0; a < Q; ++a) f[i][a] = (T)fsrc[(i * Q + a) * ns_ + node];
        } else {
            const T n = nf ? (T)nf[node] : (T)1;
            static_for<0, NS>([&](auto ic) {
                constexpr int I = decltype(ic)::value;
                const T r = (T)xf[I * ns_ + node] * p.M[I] * n;
                static_for<0, Q>([&](auto ac) {
                    constexpr int A = decltype(ac)::value;
                    const T eg = edot<LAT, A>(gn);
                    f[I][A] = p.wl[wclass<LAT>(A)] * r * ((T)1 - (T)0.5 * p.c_inv_cs2[I] * eg);
                });
            });
        }
        T R0[NS];
        to_deviations<LAT, NS, S>(p, f, R0);
        moments<LAT, NS, dev_arith<S>()>(p, f, s, err, gn, R0);
        store_all<LAT, NS>(p, fprev, node, f, s.rho, R0);
        collide<LAT, NS, dev_arith<S>(), false, Codec<S>::NODE>(p, f, s, gn);
        store_all<LAT, NS>(p, fcur, node, f, s.rho, R0);
        if (err) atomicOr(err_flag, err);
    }
    block_mass<NS>(s.rho, active, mass_part);
}

}  // namespace evd

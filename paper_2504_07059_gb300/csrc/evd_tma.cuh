// evd_tma.cuh -- the D3Q19 step with TMA-staged tiles (float / half storage).
//
// Work decomposition.  A CTA owns a column of TX x TY nodes in (x, y) and a
// chunk of z, with one thread per (node, species): warp w holds the 32
// x-nodes of row w % TY for species w / TY.  The CTA marches up its z-chunk.
// For every z-plane, one TMA tile copy (cp.async.bulk.tensor) per storage
// group brings the slabs of every (species, direction) plane into a ring of
// SLOTS shared-memory stages: the tile plus a one-node halo along the
// in-plane dimensions the group's directions move in.  Each stage completes
// on its own mbarrier (transaction bytes).  The copies for stage idx+SLOTS-1
// are issued by seven lanes of warp 0 at the top of iteration idx, into the
// slot every warp finished reading before the previous iteration's barrier,
// so SLOTS-1 stages are in flight while one is computed.
//
// Each slab is read once: its in-plane interpolation R (1, 3 or 3x3 points of
// Eq. Second_order_spatial_interpolation) is formed in registers, then
//   * directions without a z component keep R as the value of the node at
//     that z (delayed one iteration, so the slab need not stay resident);
//   * directions with a z component add w(oz) R to the running sums of the
//     nodes at z+1, z and z-1 (the z-part of the tensor-product weights),
//     and the node at z-1 is complete.
// So iteration k of the march finishes the node at z = k - 1.  The species of
// a node then exchange rho_i and u_i^eq through shared memory (one barrier of
// the compute warps per iteration) for the cross collision, and each thread
// collides and stores its own 19 populations.
//
// Walls: a stencil node beyond a wall reads as zero (the fill of the tile
// copy outside the lattice), so the full weights act as the weights of the
// fluid nodes alone; a z-slab beyond a z wall contributes nothing.
// Wall-adjacent nodes add the App. A lumped terms f_a += L_self f*_a(O) +
// L_opp f*_abar(O), their own populations f*(O) being the centre of the
// stage that holds their slab: the terms go into the node's running sums in
// the iteration that reads that slab (closed form at a flat wall; the host
// table of the wall class at edges and corners).
// Periodic z is a wrapped slab coordinate; x and y must be walled (other
// geometries use the general kernel).
#pragma once

#include <cuda.h>

#include "evd_device.cuh"

namespace evd {

constexpr int TTX = 32;
constexpr int NGRP = 7;       // storage groups of directions
constexpr int NGRP_MAX = 8;   // + the node-density planes of half storage (group 7)
constexpr unsigned ERR_TIMEOUT = 4u;

template <typename S> struct TmaPad;
template <> struct TmaPad<float> { static constexpr int XP = 4; };   // 16 bytes
template <> struct TmaPad<__half> { static constexpr int XP = 8; };  // 16 bytes

// halo class of a storage group: bit 0 moves in x, bit 1 moves in y (the
// node densities, group 7, are read at every in-plane stencil node)
__host__ __device__ constexpr int grp_cls(int g)
{
    return g == 2 || g == 3 ? 1 : g == 4 || g == 5 ? 2 : g == 6 || g == 7 ? 3 : 0;
}
__host__ __device__ constexpr bool grp_moves_z(int g) { return g == 1 || g == 3 || g == 5; }
// loaded for the halo z-planes too: the z-moving groups, and the node
// densities that decode them
__host__ __device__ constexpr bool grp_on_halo(int g) { return grp_moves_z(g) || g == 7; }
__host__ __device__ constexpr int grp_planes(int g) { return g == 7 ? 1 : grp_size(g); }

template <int NS, typename S, int TY, int SLOTS>
struct TmaLayout {
    static constexpr int XP = TmaPad<S>::XP;
    static constexpr int threads = TTX * TY * NS;
    static constexpr bool LOCAL = Codec<S>::LOCAL;
    static constexpr int NG = LOCAL ? NGRP + 1 : NGRP;
    static __host__ __device__ constexpr int bw(int cls) { return (cls & 1) ? TTX + 2 * XP : TTX; }
    static __host__ __device__ constexpr int bh(int cls) { return (cls & 2) ? TY + 2 : TY; }
    static __host__ __device__ constexpr int plane_elems(int g) { return bw(grp_cls(g)) * bh(grp_cls(g)); }
    static __host__ __device__ constexpr int box_bytes(int g)
    {
        return plane_elems(g) * NS * grp_planes(g) * (int)sizeof(S);
    }
    static __host__ __device__ constexpr int group_offset(int g)
    {
        int o = 0;
        for (int q = 0; q < g; ++q) o += (box_bytes(q) + 127) / 128 * 128;
        return o;
    }
    static constexpr int slot_bytes = group_offset(NG);
    static __host__ __device__ constexpr int stage_bytes(bool halo)
    {
        int s = 0;
        for (int g = 0; g < NG; ++g)
            if (!halo || grp_on_halo(g)) s += box_bytes(g);
        return s;
    }
    static constexpr int ring_bytes = SLOTS * slot_bytes;
    static constexpr int exch_bytes = 2 * NS * TY * TTX * 16;   // two float4 buffers
    static constexpr int msum_offset = ring_bytes + exch_bytes;
    static constexpr int bar_offset = msum_offset + NS * TY * 8 + 8;
    static constexpr int total_bytes = bar_offset + SLOTS * 8 + 128;   // + alignment slack
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}


__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after `polls` polls.  The step's waits take
// WAIT_POLLS (far longer than any copy takes) unless the caller lowers it.
constexpr int WAIT_POLLS = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, int polls = WAIT_POLLS)
{
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// 4-byte global -> shared copy that holds no register while in flight
__device__ __forceinline__ void cp_async4(unsigned dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct TmaMaps {
    CUtensorMap m[NGRP_MAX];   // one per storage group of the input buffer
};

// Which z-planes a stage loads: all groups for z in [zb, ze), only the
// z-moving groups (and node densities) for the halo planes zb-1 and ze.
__device__ __forceinline__ bool stage_is_halo(int k, int zb, int ze) { return k < zb || k >= ze; }

// ------------------------------------------------------ packed float pairs
// The two members of an opposite-direction pair (A, A + 1 in the library's
// D3Q19 order) go through the same operations; f32x2 instructions issue both
// at once.  Their rounding is that of the scalar operations.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// 1-D weights of source offset o (-1, 0, 1) for a pair whose first member
// moves in +e (first = true) or -e: WP[o + 1] = (W for +e, W for -e) with
// W(o; e) = w[widx(o, e)]; for the pair led by -e the members swap.
struct WPair {
    float2 w[3];   // (w[widx(o, +1)], w[widx(o, -1)]) at index o + 1
};

__device__ __forceinline__ WPair weight_pairs(const float (&w)[3])
{
    WPair p;
    p.w[0] = make_float2(w[0], w[2]);
    p.w[1] = make_float2(w[1], w[1]);
    p.w[2] = make_float2(w[2], w[0]);
    return p;
}

template <int e>
__device__ __forceinline__ float2 wpo(const WPair& p, int o)
{
    return e > 0 ? p.w[o + 1] : p.w[1 - o];
}

// Half storage: the stored densities rho~ of the 3x3 in-plane neighbourhood of
// the thread's node in this stage (group 7, which carries the x and y halo;
// nodes beyond a wall read as zero, the fill of the tile copy).
template <int NS, typename S, int TY, int SLOTS>
__device__ __forceinline__ void dens_block(const unsigned char* slot, int sp, int tx, int ty, float (&rd)[3][3])
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int W7 = G::bw(3);
    const S* r = reinterpret_cast<const S*>(slot + G::group_offset(7)) + sp * G::plane_elems(7);
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) rd[oy][ox] = (float)r[(ty + oy) * W7 + tx + G::XP - 1 + ox];
}

// rho~ interpolated with the in-plane stencil of the directions whose
// in-plane components are (ex, ey).  A half population is g + w_a rho~ at
// every stencil node, so by linearity its interpolant is the interpolant of
// g plus w_a times this one, which every direction with the same (ex, ey)
// shares (up to three in D3Q19).
template <int ex, int ey>
__device__ __forceinline__ float dens_interp(const float (&rd)[3][3], const float (&w)[3])
{
    auto row = [&](int oy) -> float {
        if constexpr (ex == 0) return rd[oy][1];
        else return w[widx(1, ex)] * rd[oy][2] + (w[widx(0, ex)] * rd[oy][1] + w[widx(-1, ex)] * rd[oy][0]);
    };
    if constexpr (ey == 0) return row(1);
    else return w[widx(1, ey)] * row(2) + (w[widx(0, ey)] * row(1) + w[widx(-1, ey)] * row(0));
}

// In-plane interpolation of the pair (A, A + 1) of one slab: the 1, 3 or 3x3
// points of Eq. Second_order_spatial_interpolation in the slab's plane, the
// two members' planes being adjacent in the stage.  A stencil node beyond a
// wall holds zero (the tile copy's fill), so the full weights act as the
// weights of the fluid nodes alone.  Float storage interpolates the
// deviations from its reference as they are (the reference carried by the
// weights is added at wall nodes only, through K - 1); half storage adds
// w_a times dI, the interpolated node densities of each member's stencil.
template <int A, int NS, typename S, int TY, int SLOTS>
__device__ __forceinline__ float2 inplane2(const unsigned char* slot, int sp, int tx, int ty, const WPair& wp,
                                           float2 dI, float wa)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int ex = ev<1>(A, 0), ey = ev<1>(A, 1);
    constexpr int g = grp<1>(A);
    constexpr int cls = grp_cls(g);
    constexpr int W = G::bw(cls);
    constexpr int PE = G::plane_elems(g);
    static_assert(grp_pos<1>(A + 1) == grp_pos<1>(A) + 1 && opp<1>(A) == A + 1, "pair planes must be adjacent");
    const S* s = reinterpret_cast<const S*>(slot + G::group_offset(g)) + (sp * grp_size(g) + grp_pos<1>(A)) * PE;
    const int cx = tx + ((cls & 1) ? G::XP : 0);
    const int cy = ty + ((cls & 2) ? 1 : 0);
    auto ld = [&](int yy, int xx) -> float2 {
        return make_float2((float)s[yy * W + xx], (float)s[PE + yy * W + xx]);
    };
    auto xrow = [&](int yy) -> float2 {
        return pfma(wpo<ex>(wp, 1), ld(yy, cx + 1), pfma(wpo<ex>(wp, 0), ld(yy, cx), pmul(wpo<ex>(wp, -1), ld(yy, cx - 1))));
    };
    float2 v;
    if constexpr (cls == 0) {
        v = ld(cy, cx);
    } else if constexpr (cls == 1) {
        v = xrow(cy);
    } else if constexpr (cls == 2) {
        v = pfma(wpo<ey>(wp, 1), ld(cy + 1, cx), pfma(wpo<ey>(wp, 0), ld(cy, cx), pmul(wpo<ey>(wp, -1), ld(cy - 1, cx))));
    } else {
        v = pfma(wpo<ey>(wp, 1), xrow(cy + 1), pfma(wpo<ey>(wp, 0), xrow(cy), pmul(wpo<ey>(wp, -1), xrow(cy - 1))));
    }
    if constexpr (G::LOCAL) return pfma(bc2(wa), dI, v);
    else return v;
}

// The stored value of direction A at the thread's own node in this stage's
// tile (the centre of its stencil; half storage: not decoded).
template <int A, int NS, typename S, int TY, int SLOTS>
__device__ __forceinline__ float tile_center(const unsigned char* slot, int sp, int tx, int ty)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int g = grp<1>(A);
    constexpr int cls = grp_cls(g);
    constexpr int W = G::bw(cls);
    const S* s = reinterpret_cast<const S*>(slot + G::group_offset(g)) +
                 (sp * grp_size(g) + grp_pos<1>(A)) * G::plane_elems(g);
    return (float)s[(ty + ((cls & 2) ? 1 : 0)) * W + tx + ((cls & 1) ? G::XP : 0)];
}

// Unit lattice speed: weights (1, 0, 0), each member's upstream node (half
// storage: dI is that node's density rho~); a node beyond a wall reads zero.
template <int A, int NS, typename S, int TY, int SLOTS>
__device__ __forceinline__ float inplane_unit(const unsigned char* slot, int sp, int tx, int ty, float dI, float wa)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int ex = ev<1>(A, 0), ey = ev<1>(A, 1);
    constexpr int g = grp<1>(A);
    constexpr int cls = grp_cls(g);
    constexpr int W = G::bw(cls);
    const S* s = reinterpret_cast<const S*>(slot + G::group_offset(g)) +
                 (sp * grp_size(g) + grp_pos<1>(A)) * G::plane_elems(g);
    const int cx = tx + ((cls & 1) ? G::XP : 0) - ex;
    const int cy = ty + ((cls & 2) ? 1 : 0) - ey;
    if constexpr (G::LOCAL) return fmaf(wa, dI, (float)s[cy * W + cx]);
    else return (float)s[cy * W + cx];
}

// e_A . v for the unit vector of direction A, starting from its first term
template <int A>
__device__ __forceinline__ float edot3(const float (&v)[3])
{
    return edot<1, A>(v);
}

// App. A terms of a node at an edge or corner (two or three walls) from the
// host table of its wall class: t[a - 1] = L_self f*_a + L_opp f*_abar (+ the
// reference the weights carry, float storage) for a = 1..18, f* the node's own
// populations in this stage's tile (half storage: decoded with the node's
// density rdc).  Out of line: such nodes are rare, and inlined, the table
// loads would be scheduled early and hold registers across the interpolation.
template <int NS, typename S, int TY, int SLOTS>
__device__ __noinline__ void wall_terms_table(const unsigned char* base, int sp, int tx, int ty,
                                              const float4* __restrict__ L, float ref1, float ref2, float wl1,
                                              float wl2, float rdc, float* __restrict__ t)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    static_for<0, 9>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int A = 2 * K + 1, B = A + 1;
        constexpr bool diag = wclass<1>(A) == 2;
        const float4 la = __ldg(L + A), lb = __ldg(L + B);
        float ca = tile_center<A, NS, S, TY, SLOTS>(base, sp, tx, ty);
        float cb = tile_center<B, NS, S, TY, SLOTS>(base, sp, tx, ty);
        float ref = 0.0f;
        if constexpr (G::LOCAL) {
            ca = fmaf(diag ? wl2 : wl1, rdc, ca);
            cb = fmaf(diag ? wl2 : wl1, rdc, cb);
        } else {
            ref = diag ? ref2 : ref1;
        }
        t[A - 1] = la.x * ca + la.y * cb + ref * la.z;
        t[B - 1] = lb.x * cb + lb.y * ca + ref * lb.z;
    });
}

template <int NS, typename S, int TY, int SLOTS>
__global__ void __launch_bounds__(TmaLayout<NS, S, TY, SLOTS>::threads, TY == 1 ? 5 : (TY == 2 ? 2 : 1))
k_step_tma(const __grid_constant__ TmaMaps maps, const Params<float> p, const S* __restrict__ fin,
           S* __restrict__ fout, double* __restrict__ mass_part, unsigned* __restrict__ err_flag, int flags,
           const double* __restrict__ corr, const float4* __restrict__ lumps, int ntx, int nty, int zchunk,
           int wait_polls)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int Q = 19;
    constexpr int NP = 9;   // opposite-direction pairs (2k + 1, 2k + 2)
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    float4* exch = reinterpret_cast<float4*>(smem + G::ring_bytes);
    double* msum = reinterpret_cast<double*>(smem + G::msum_offset);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + G::bar_offset);
    const unsigned ring = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x % (ntx * nty);
    const int chunk = blockIdx.x / (ntx * nty);
    const int x0 = (tile % ntx) * TTX, y0 = (tile / ntx) * TY;
    const int zb = chunk * zchunk;
    const int ze = min(zb + zchunk, p.nz);
    const int zwall = p.wall[2];
    const int kfirst = zb - 1;
    const int nstage = ze - zb + 2;   // stages k = zb-1 .. ze

    if (threadIdx.x == 0) {
        for (int s = 0; s < SLOTS; ++s) mbar_init(full(s), 1);
        fence_mbar_init();
    }
    __syncthreads();

    // copy parameters of the storage group this lane of warp 0 issues
    const int g = lane < G::NG ? lane : 0;
    const int gcls = grp_cls(g);
    const int gcx = (gcls & 1) ? x0 - G::XP : x0;
    const int gcy = (gcls & 2) ? y0 - 1 : y0;
    const int gc3 = g == 7 ? NS * 19 : NS * grp_start(g);   // group 7: the node densities
    const unsigned goff = (unsigned)G::group_offset(g);
    const bool gz = grp_on_halo(g);
    const bool issuer = warp == 0 && lane < G::NG;
    auto issue = [&](int idx) {
        const int slot = idx % SLOTS;
        const int k = kfirst + idx;
        const bool halo = stage_is_halo(k, zb, ze);
        // walled z: a slab beyond the wall is out of range and reads as zero
        const int zc = zwall ? k : (k % p.nz + p.nz) % p.nz;
        if (lane == 0) mbar_arrive_expect_tx(full(slot), (unsigned)G::stage_bytes(halo));
        if (!halo || gz) tma_load_4d(ring + (unsigned)(slot * G::slot_bytes) + goff, &maps.m[g], gcx, gcy, zc, gc3,
                                     full(slot));
    };
    if (issuer)
        for (int idx = 0; idx < SLOTS - 1 && idx < nstage; ++idx) issue(idx);

    // ------------------------------------------------------------ compute
    const int ty = warp % TY, sp = warp / TY;
    const int tx = lane;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) w[a] = p.w1[sp][a];
    const WPair wp = weight_pairs(w);
    const float csp = p.c[sp], inv_cs2 = p.inv_cs2[sp], c_inv_cs2 = p.c_inv_cs2[sp], c_inv_lo = p.c_inv_cs2_lo[sp];
    const float tau_inv = p.tau_inv[sp], omt = p.omt[sp];
    const float isf = inv_cs2 * p.sfac[sp];
    const bool xlo = p.wall[0] && x == 0, xhi = p.wall[0] && x == p.nx - 1;
    const bool ylo = p.wall[1] && y == 0, yhi = p.wall[1] && y == p.ny - 1;
    const bool col_wall = xlo || xhi || ylo || yhi;
    const int wcls_xy = (xlo ? 1 : (xhi ? 2 : 0)) + 3 * (ylo ? 1 : (yhi ? 2 : 0));
    const bool unit = p.unit[sp] != 0;   // the same for the whole warp
    const int nxy = p.nx * p.ny;
    const int pstride = (int)p.pstride;   // the host guarantees planes * pstride < 2^31
    const bool want_mass = (flags & F_MASS) != 0;

    // running sums, per pair k: z-moving pairs (A: node at z = k-1, B: node
    // at k), in-plane pairs and the rest (N: value at z = k-1)
    float2 accA[NP], accB[NP], accN[NP];
    float accN0 = 0.0f;
#pragma unroll
    for (int k = 0; k < NP; ++k) accA[k] = accB[k] = accN[k] = make_float2(0.0f, 0.0f);
    double mass_acc = 0.0;
    unsigned err = 0;
    bool failed = false;
    int fail_idx = 0;   // iteration whose wait gave up

    for (int idx = 0; idx < nstage; ++idx) {
        const int k = kfirst + idx;
        const int slot = idx % SLOTS;
        if (issuer && idx + SLOTS - 1 < nstage) {
            // the slot of stage idx-1, read by every warp before the last barrier
            fence_proxy_async();
            issue(idx + SLOTS - 1);
        }
        const unsigned char* base = smem + slot * G::slot_bytes;
        const bool halo = stage_is_halo(k, zb, ze);
        const int zo = k - 1;                   // node finished this iteration
        const bool emit = zo >= zb && zo < ze;  // the same for every thread of the CTA
        const int node = x + p.nx * y + nxy * zo;
        // the node of this stage's slab, finished next iteration, at a wall
        const bool wall_next = !halo && active && (col_wall || (zwall && (k == 0 || k == p.nz - 1)));
        const bool ok = mbar_wait_bounded(full(slot), (unsigned)((idx / SLOTS) & 1), wait_polls);
        // half storage: this stage's node densities around the node (the
        // density term of every stencil is taken from them once per stage)
        float rd[3][3] = {};
        if constexpr (G::LOCAL)
            if (ok) dens_block<NS, S, TY, SLOTS>(base, sp, tx, ty, rd);
        float f0 = accN0;
        float2 F[NP];
        if (ok) {
            // The same running sums for every species; a unit-speed species
            // (c = 1, weights (1, 0, 0)) reads each member's upstream node
            // instead of interpolating (exact shift), and its z sums multiply
            // by exactly one and zero.
            float di[3][3] = {};   // [ey + 1][ex + 1]
            if constexpr (G::LOCAL)
                if (!unit)
                    static_for<0, 9>([&](auto kc) {
                        constexpr int K = decltype(kc)::value;
                        di[K / 3][K % 3] = dens_interp<K % 3 - 1, K / 3 - 1>(rd, w);
                    });
            if (!halo) {
                if constexpr (G::LOCAL) accN0 = inplane_unit<0, NS, S, TY, SLOTS>(base, sp, tx, ty, rd[1][1], p.wl[0]);
                else accN0 = inplane_unit<0, NS, S, TY, SLOTS>(base, sp, tx, ty, 0.0f, 0.0f);
            }
            auto march = [&](auto uc) {
                constexpr bool UNIT = decltype(uc)::value;
                static_for<0, NP>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    constexpr int A = 2 * K + 1, B = A + 1;
                    constexpr int ex = ev<1>(A, 0), ey = ev<1>(A, 1), ez = ev<1>(A, 2);
                    const float wa = p.wl[wclass<1>(A)];
                    auto slab = [&]() -> float2 {   // this slab's in-plane value of the pair
                        if constexpr (UNIT)
                            return make_float2(inplane_unit<A, NS, S, TY, SLOTS>(base, sp, tx, ty, rd[1 - ey][1 - ex], wa),
                                               inplane_unit<B, NS, S, TY, SLOTS>(base, sp, tx, ty, rd[1 + ey][1 + ex], wa));
                        else
                            return inplane2<A, NS, S, TY, SLOTS>(base, sp, tx, ty, wp,
                                                                 make_float2(di[ey + 1][ex + 1], di[1 - ey][1 - ex]), wa);
                    };
                    if constexpr (ez == 0) {
                        F[K] = accN[K];
                        if (!halo) accN[K] = slab();
                    } else {
                        const float2 R = slab();
                        // slab k feeds the nodes at z = k+1 (oz=-1), k (0), k-1 (+1)
                        F[K] = pfma(wpo<ez>(wp, 1), R, accA[K]);
                        accA[K] = pfma(wpo<ez>(wp, 0), R, accB[K]);
                        accB[K] = pmul(wpo<ez>(wp, -1), R);
                    }
                });
            };
            if (unit) march(std::true_type{});
            else march(std::false_type{});
        }
        // App. A terms of the wall node of this slab (finished next
        // iteration), from its own post-collision populations, which are the
        // centre of every plane of this stage's tile: L_self f*_a + L_opp
        // f*_abar (+ the reference the weights carry, float storage), added
        // to the node's running sums (accN: in-plane pairs, accA: z-moving).
        if (ok && wall_next) {
            const bool zw = zwall && (k == 0 || k == p.nz - 1);
            const bool xw = xlo || xhi, yw = ylo || yhi;
            auto add_term = [&](auto kc, float2 v) {
                constexpr int K = decltype(kc)::value;
                if constexpr (ev<1>(2 * K + 1, 2) == 0) accN[K] = padd(accN[K], v);
                else accA[K] = padd(accA[K], v);
            };
            if ((int)xw + (int)yw + (int)zw == 1) {
                // one flat wall (the common case): with w = (w0, w1, w2) the
                // species' 1-D weights, a direction moving away from the wall
                // keeps its own weight w2 that crossed it (L_self = w2), takes
                // its opposite's crossing weight w0 (L_opp = w0), and carries
                // K - 1 = w2; the direction heading into the wall carries
                // K - 1 = -w2; directions along the wall have none.  The host
                // table holds the same coefficients for every wall class.
                const int kd = xw ? 0 : (yw ? 1 : 2);
                const bool at_hi = xw ? xhi : (yw ? yhi : k == p.nz - 1);
                const float w0 = w[0], w2 = w[2];
                static_for<0, NP>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    constexpr int A = 2 * K + 1, B = A + 1;
                    const int e = kd == 0 ? ev<1>(A, 0) : (kd == 1 ? ev<1>(A, 1) : ev<1>(A, 2));
                    const int away = at_hi ? -e : e;   // +1: A leaves the wall, -1: A heads into it
                    if (away != 0) {
                        float ca = tile_center<A, NS, S, TY, SLOTS>(base, sp, tx, ty);
                        float cb = tile_center<B, NS, S, TY, SLOTS>(base, sp, tx, ty);
                        float ref = 0.0f;
                        if constexpr (G::LOCAL) {   // decoded with the node's density
                            ca = fmaf(p.wl[wclass<1>(A)], rd[1][1], ca);
                            cb = fmaf(p.wl[wclass<1>(A)], rd[1][1], cb);
                        } else {
                            ref = p.ref[sp][wclass<1>(A)];
                        }
                        const float2 t = away > 0 ? make_float2(w2 * ca + w0 * cb + ref * w2, ref * -w2)
                                                  : make_float2(ref * -w2, w2 * cb + w0 * ca + ref * w2);
                        add_term(kc, t);
                    }
                });
            } else {   // edges and corners: the host table of the wall class
                const int zc_next = zwall ? (k == 0 ? 1 : (k == p.nz - 1 ? 2 : 0)) : 0;
                float t[18];
                wall_terms_table<NS, S, TY, SLOTS>(base, sp, tx, ty, lumps + ((wcls_xy + 9 * zc_next) * NS + sp) * Q,
                                                   p.ref[sp][1], p.ref[sp][2], p.wl[1], p.wl[2], rd[1][1], t);
                static_for<0, NP>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    add_term(kc, make_float2(t[2 * K], t[2 * K + 1]));
                });
            }
        }

        // ---- node (x, y, zo): correction, moments
        float rho = 1.0f, drho = 0.0f, ueq[3] = {0.0f, 0.0f, 0.0f};
        if (ok && emit) {
            // moments from the pairs: s = f_A + f_B adds to rho, d = f_A - f_B
            // to the momentum along A's components (sums start from a term)
            float r = f0, j[3];
            static_for<0, NP>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                constexpr int A = 2 * K + 1;
                const float sK = F[K].x + F[K].y, dK = F[K].x - F[K].y;
                r += sK;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    constexpr int first[3] = {first_dir<1>(0), first_dir<1>(1), first_dir<1>(2)};
                    const int e = ev<1>(A, d);
                    if (A == first[d]) j[d] = e > 0 ? dK : -dK;
                    else if (e == 1) j[d] += dK;
                    else if (e == -1) j[d] -= dK;
                }
            });
            drho = r;
            if (corr) {
                // mass correction in proportion to the node's density: f_a +=
                // w_a ci (ci = corr rho), which adds ci to rho and no momentum
                const float ci = (float)__ldg(corr + sp) * (Codec<S>::DARITH ? p.rref[sp] + r : r);
                drho += ci;
                f0 = fmaf(p.wl[0], ci, f0);
                const float2 c1 = bc2(p.wl[1] * ci), c2 = bc2(p.wl[2] * ci);
                static_for<0, NP>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    F[K] = padd(F[K], wclass<1>(2 * K + 1) == 1 ? c1 : c2);
                });
            }
            r = Codec<S>::DARITH ? p.rref[sp] + drho : drho;
            if (active && !(r > 0.0f)) err |= ERR_RHO;
            rho = r;
            const float rinv = __fdividef(1.0f, r);
#pragma unroll
            for (int d = 0; d < 3; ++d) ueq[d] = csp * j[d] * rinv + 0.5f * p.g[d];
            exch[((idx & 1) * NS * TY + sp * TY + ty) * TTX + tx] = make_float4(rho, ueq[0], ueq[1], ueq[2]);
        }
        // one barrier per iteration: the exchange, the release of the stage
        // just read, and agreement on a failed wait
        failed = __syncthreads_or(!ok);
        if (failed) { fail_idx = idx; break; }
        if (!emit) continue;

        // ---- species coupling (every thread of the node recomputes it)
        float r[NS], ue[NS][3];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const float4 v = exch[((idx & 1) * NS * TY + i * TY + ty) * TTX + tx];
            r[i] = v.x; ue[i][0] = v.y; ue[i][1] = v.z; ue[i][2] = v.w;
        }
        // this thread's own rho and u^eq come back from the exchange (the same
        // values), so that they need not stay in registers across the barrier
        rho = r[0];
        ueq[0] = ue[0][0]; ueq[1] = ue[0][1]; ueq[2] = ue[0][2];
#pragma unroll
        for (int i = 1; i < NS; ++i)
            if (i == sp) { rho = r[i]; ueq[0] = ue[i][0]; ueq[1] = ue[i][1]; ueq[2] = ue[i][2]; }
        float rho_m = r[0], n = r[0] * p.Minv[0];
#pragma unroll
        for (int i = 1; i < NS; ++i) { rho_m += r[i]; n = fmaf(r[i], p.Minv[i], n); }
        const float rinv_m = __fdividef(1.0f, rho_m);
        float u[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = r[0] * ue[0][d];
#pragma unroll
            for (int i = 1; i < NS; ++i) acc = fmaf(r[i], ue[i][d], acc);
            u[d] = acc * rinv_m;
        }
        float X[MAXS][MAXS] = {};
        if constexpr (NS == 2) {
            const float A12 = (r[0] + r[1]) * p.iD[0][1] + n * p.MM[0][1];
            X[0][1] = X[1][0] = __fdividef(2.0f * rho_m * p.iD[0][1], A12);
        } else if constexpr (NS == 3) {
            const float A12 = (r[0] + r[1]) * p.iD[0][1] + n * p.MM[0][1];
            const float A13 = (r[0] + r[2]) * p.iD[0][2] + n * p.MM[0][2];
            const float A23 = (r[1] + r[2]) * p.iD[1][2] + n * p.MM[1][2];
            const float B12 = 2.0f * rho_m * p.iD[0][1];
            const float B13 = 2.0f * rho_m * p.iD[0][2];
            const float B23 = 2.0f * rho_m * p.iD[1][2];
            const float rA13 = __fdividef(1.0f, A13);
            const float X23 = __fdividef(B23 - r[0] * B13 * rA13 * p.iD[1][2],
                                         A23 - r[0] * r[1] * rA13 * p.iD[0][2] * p.iD[1][2]);
            X[0][1] = X[1][0] = __fdividef(B12 - r[2] * X23 * p.iD[0][1], A12);
            X[0][2] = X[2][0] = (B13 - r[1] * X23 * p.iD[0][2]) * rA13;
            X[1][2] = X[2][1] = X23;
        }
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int jj = i + 1; jj < NS; ++jj)
                if (active && (!(X[i][jj] > 0.0f) || !isfinite(X[i][jj]))) err |= ERR_TAU;
        // this thread's row of 1/tau_ij, weighted by rho_j / rho
        float xr[NS];
#pragma unroll
        for (int jj = 0; jj < NS; ++jj) {
            float xs = X[0][jj];
#pragma unroll
            for (int i = 1; i < NS; ++i) xs = (i == sp) ? X[i][jj] : xs;
            xr[jj] = (jj == sp) ? 0.0f : r[jj] * xs * rinv_m;
        }
        float V[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = xr[0] * (ueq[d] - ue[0][d]);
#pragma unroll
            for (int jj = 1; jj < NS; ++jj) acc = fmaf(xr[jj], ueq[d] - ue[jj][d], acc);
            V[d] = acc;
        }

        // ---- collision of this species (Eq. LBE_forcing), pairs at a time.
        // With t = c e.u/cs^2, b = c e.a/cs^2 (a = (u^eq - u)/tau - V),
        // gam = c e.g, all odd in e, and P = t^2/2 + U2 even, a pair (A, -A)
        // updates as  f*_+- = omt f_+- + E +- O  with
        //   half  (f):  E = w rho (P T + t b) + K (gam t - u.g),
        //               O = w rho (t T + b P) + K gam,
        //               T = 1/tau - (u.a)/cs^2, U2 = 1 - u^2/(2 cs^2);
        //   float (deviations g = f - ref):
        //               E = w rho (P T + t b + Bm) + K (gam t - u.g) + (w drho + refc)/tau,
        //               O = w rho (t T + b (P + 1)) + K gam,
        //               Bm = -(u.a)/cs^2, U2 = -u^2/(2 cs^2);
        //   K = w rho (1 - 1/(2 tau))/cs^2.
        constexpr bool DA = Codec<S>::DARITH;
        float av[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) av[d] = fmaf(ueq[d] - u[d], tau_inv, -V[d]);
        const float ua = fmaf(u[2], av[2], fmaf(u[1], av[1], u[0] * av[0]));
        const float usq = fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));
        const float ug = fmaf(u[2], p.g[2], fmaf(u[1], p.g[1], u[0] * p.g[0]));
        const float Bm = -inv_cs2 * ua;
        const float T = tau_inv + Bm;
        const float U2 = DA ? -0.5f * inv_cs2 * usq : fmaf(-0.5f * inv_cs2, usq, 1.0f);
        float U[3], Av[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {   // k = c / c_s^2 as k_hi + k_lo: exact species momentum
            U[d] = fmaf(c_inv_cs2, u[d], c_inv_lo * u[d]);
            Av[d] = fmaf(c_inv_cs2, av[d], c_inv_lo * av[d]);
        }
        const float sr = rho * isf;
        float wr[3], Kc[3], Cc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            wr[c] = p.wl[c] * rho;
            Kc[c] = p.wl[c] * sr;
            const float dtt = DA ? fmaf(p.wl[c], drho, p.refc[sp][c]) * tau_inv : 0.0f;   // (w rho - ref)/tau
            Cc[c] = fmaf(-Kc[c], ug, dtt);
        }
        if (active && want_mass) mass_acc += (double)rho;
        // half storage: the node density, rounded as stored, is the reference
        float rr = 0.0f;
        if constexpr (G::LOCAL) {
            rr = Codec<S>::rt(rho);
            if (active) Codec<S>::st(fout + (ref_plane<1, NS>(sp) * pstride + node), rr);
        }
        auto store = [&](int A, int C, float fs) {
            if (active) {
                if constexpr (G::LOCAL) Codec<S>::st(fout + (plane_of<1, NS>(sp, A) * pstride + node), fs - p.wl[C] * rr);
                else Codec<S>::st(fout + (plane_of<1, NS>(sp, A) * pstride + node), fs);
            }
        };
        {   // rest: t = b = gam = 0
            const float XE0 = DA ? fmaf(U2, T, Bm) : U2 * T;
            store(0, 0, fmaf(omt, f0, fmaf(wr[0], XE0, Cc[0])));
        }
        static_for<0, NP>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            constexpr int A = 2 * K + 1;
            constexpr int C = wclass<1>(A);
            const float t = edot3<A>(U), b = edot3<A>(Av), gam = csp * edot3<A>(p.g);
            const float P = fmaf(0.5f * t, t, U2);
            const float XE = DA ? fmaf(P, T, fmaf(t, b, Bm)) : fmaf(P, T, t * b);
            const float XO = DA ? fmaf(t, T, fmaf(b, P, b)) : fmaf(t, T, b * P);
            const float Kg = Kc[C] * gam;
            const float E = fmaf(wr[C], XE, fmaf(Kg, t, Cc[C]));
            const float O = fmaf(wr[C], XO, Kg);
            const float2 fs = pfma(bc2(omt), F[K], pfma(make_float2(1.0f, -1.0f), bc2(O), bc2(E)));
            store(A, C, fs.x);
            store(A + 1, C, fs.y);
        });
    }

    if (failed) {
        // never expected: report, let every copy still in flight land in this
        // CTA's shared memory, and leave.  In flight are the stages issued up
        // to iteration fail_idx: fail_idx .. fail_idx + SLOTS - 1 (those that
        // exist); stage s completes phase s / SLOTS of the barrier of slot
        // s % SLOTS, so each is waited for with that phase's parity (a stage
        // that already landed returns at once).  These waits always take the
        // full poll count.
        if (threadIdx.x == 0) {
            atomicOr(err_flag, ERR_TIMEOUT);
            const int last = min(fail_idx + SLOTS - 1, nstage - 1);
            for (int s = fail_idx; s <= last; ++s)
                (void)mbar_wait_bounded(full(s % SLOTS), (unsigned)((s / SLOTS) & 1), WAIT_POLLS);
        }
        __syncthreads();
        return;
    }
    if (err) atomicOr(err_flag, err);
    if (want_mass) {
        // per-species block partial over the TY warps of a species, fixed order
        double v = mass_acc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) msum[sp * TY + ty] = v;
        __syncthreads();
        if (threadIdx.x < NS) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < TY; ++q) t += msum[threadIdx.x * TY + q];
            mass_part[(long long)blockIdx.x * NS + threadIdx.x] = t;
        }
    }
}

}  // namespace evd

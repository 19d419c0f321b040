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
// Walls: a thread's (x, y) column is fixed for the whole march, so solid
// in-plane stencil nodes are removed once, by zeroing their weights; a z-slab
// beyond a z wall contributes nothing.  Wall-adjacent nodes add the App. A
// lumped terms f_a += L_self f*_a(O) + L_opp f*_abar(O), with the coefficients
// of their wall class (which of the six walls they touch) from a table built
// on the host, and their own populations f*(O) fetched from global memory at
// the start of the iteration so that the loads overlap the interpolation.
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
    // float storage: wall populations of the node land here by cp.async
    // ([direction][thread] words) instead of in registers
    static constexpr bool CEN_SMEM = sizeof(S) == 4;
    static constexpr int cen_offset = ring_bytes + exch_bytes;
    static constexpr int cen_bytes = CEN_SMEM ? 19 * threads * 4 : 0;
    static constexpr int msum_offset = cen_offset + cen_bytes;
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

// masked 1-D weights of one in-plane dimension for a direction component e
// (+1 -> index 0, -1 -> index 1): solid stencil nodes get weight zero
struct MaskedW {
    float w[2][3];
    float sum[2];
};

__device__ __forceinline__ MaskedW masked_weights(const float (&w)[3], bool lo, bool hi)
{
    MaskedW m;
#pragma unroll
    for (int ei = 0; ei < 2; ++ei) {
        const int e = ei == 0 ? 1 : -1;
        float s = 0.0f;
#pragma unroll
        for (int o = -1; o <= 1; ++o) {
            const bool solid = (o == -1 && lo) || (o == 1 && hi);
            const float v = solid ? 0.0f : w[o == -e ? 0 : (o == 0 ? 1 : 2)];
            m.w[ei][o + 1] = v;
            s += v;
        }
        m.sum[ei] = s;
    }
    return m;
}

// Half storage: the stored densities rho~ of the 3x3 in-plane neighbourhood of
// the thread's node in this stage (group 7, which carries the x and y halo).
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

// rho~ interpolated with the in-plane stencil (and masked weights) of the
// directions whose in-plane components are (ex, ey).  A half population is
// g + w_a rho~ at every stencil node, so by linearity its interpolant is the
// interpolant of g plus w_a times this one, which every direction with the
// same (ex, ey) shares (up to three in D3Q19).
template <int ex, int ey>
__device__ __forceinline__ float dens_interp(const float (&rd)[3][3], const MaskedW& mx, const MaskedW& my)
{
    constexpr int xi = ex > 0 ? 0 : 1, yi = ey > 0 ? 0 : 1;
    auto row = [&](int oy) -> float {
        if constexpr (ex == 0) return rd[oy][1];
        else return mx.w[xi][0] * rd[oy][0] + mx.w[xi][1] * rd[oy][1] + mx.w[xi][2] * rd[oy][2];
    };
    if constexpr (ey == 0) return row(1);
    else return my.w[yi][0] * row(0) + my.w[yi][1] * row(1) + my.w[yi][2] * row(2);
}

// In-plane interpolation of direction A: float storage interpolates the
// deviations from its reference as they are (the reference carried by the
// weights is added at wall nodes only, through K - 1); half storage
// interpolates the stored g and adds wa times dI, the interpolated node
// densities of the direction's stencil (dens_interp).
template <int A, int NS, typename S, int TY, int SLOTS>
__device__ __forceinline__ float inplane(const unsigned char* slot, int sp, int tx, int ty, const MaskedW& mx,
                                         const MaskedW& my, float dI, float wa)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int ex = ev<1>(A, 0), ey = ev<1>(A, 1);
    constexpr int g = grp<1>(A);
    constexpr int cls = grp_cls(g);
    constexpr int W = G::bw(cls);
    constexpr int xi = ex > 0 ? 0 : 1, yi = ey > 0 ? 0 : 1;
    const S* s = reinterpret_cast<const S*>(slot + G::group_offset(g)) +
                 (sp * grp_size(g) + grp_pos<1>(A)) * G::plane_elems(g);
    const int cx = tx + ((cls & 1) ? G::XP : 0);
    const int cy = ty + ((cls & 2) ? 1 : 0);
    auto ld = [&](int yy, int xx) -> float { return (float)s[yy * W + xx]; };
    float v;
    if constexpr (cls == 0) {
        v = ld(cy, cx);
    } else if constexpr (cls == 1) {
        v = mx.w[xi][0] * ld(cy, cx - 1) + mx.w[xi][1] * ld(cy, cx) + mx.w[xi][2] * ld(cy, cx + 1);
    } else if constexpr (cls == 2) {
        v = my.w[yi][0] * ld(cy - 1, cx) + my.w[yi][1] * ld(cy, cx) + my.w[yi][2] * ld(cy + 1, cx);
    } else {
        float acc = 0.0f;
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy) {
            const float row = mx.w[xi][0] * ld(cy + oy, cx - 1) + mx.w[xi][1] * ld(cy + oy, cx) +
                              mx.w[xi][2] * ld(cy + oy, cx + 1);
            acc += my.w[yi][oy + 1] * row;
        }
        v = acc;
    }
    if constexpr (G::LOCAL) return fmaf(wa, dI, v);
    else return v;
}

// Unit lattice speed off the walls: weights (1, 0, 0), the upstream node
// (half storage: dI is that node's density rho~).
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

template <int NS, typename S, int TY, int SLOTS>
__global__ void __launch_bounds__(TmaLayout<NS, S, TY, SLOTS>::threads, TY == 2 ? 2 : 1)
k_step_tma(const __grid_constant__ TmaMaps maps, const Params<float> p, const S* __restrict__ fin,
           S* __restrict__ fout, double* __restrict__ mass_part, unsigned* __restrict__ err_flag, int flags,
           const double* __restrict__ corr, const float4* __restrict__ lumps, int ntx, int nty, int zchunk,
           int wait_polls)
{
    using G = TmaLayout<NS, S, TY, SLOTS>;
    constexpr int Q = 19;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    float4* exch = reinterpret_cast<float4*>(smem + G::ring_bytes);
    double* msum = reinterpret_cast<double*>(smem + G::msum_offset);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + G::bar_offset);
    const unsigned ring = smem_u32(smem);
    const unsigned cen_s = smem_u32(smem + G::cen_offset);
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
        const int zc = zwall ? k : (k % p.nz + p.nz) % p.nz;   // walled: out of range -> zero fill
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
    const float csp = p.c[sp], inv_cs2 = p.inv_cs2[sp], c_inv_cs2 = p.c_inv_cs2[sp];
    const float tau_inv = p.tau_inv[sp], omt = p.omt[sp], sfac = p.sfac[sp];
    const bool xlo = p.wall[0] && x == 0, xhi = p.wall[0] && x == p.nx - 1;
    const bool ylo = p.wall[1] && y == 0, yhi = p.wall[1] && y == p.ny - 1;
    const bool col_wall = xlo || xhi || ylo || yhi;
    const MaskedW mx = masked_weights(w, xlo, xhi), my = masked_weights(w, ylo, yhi);
    const bool unit_fast = p.unit[sp] && !col_wall;
    const int nxy = p.nx * p.ny;
    const int pstride = (int)p.pstride;   // the host guarantees planes * pstride < 2^31
    const int wcls_xy = (xlo ? 1 : (xhi ? 2 : 0)) + 3 * (ylo ? 1 : (yhi ? 2 : 0));

    // running sums: z-moving directions (A: node at z = k-1, B: node at k),
    // in-plane directions (N: value at z = k-1)
    float accA[Q], accB[Q], accN[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) accA[a] = accB[a] = accN[a] = 0.0f;
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
        const bool solid_slab = zwall && (k < 0 || k >= p.nz);
        const int zo = k - 1;                   // node finished this iteration
        const bool emit = zo >= zb && zo < ze;  // the same for every thread of the CTA
        const bool zlo = zwall && zo == 0, zhi = zwall && zo == p.nz - 1;
        const int node = x + p.nx * y + nxy * zo;
        const bool wall_node = emit && active && (col_wall || zlo || zhi);
        float f[Q], cen[Q], cenr = 0.0f;
        if (wall_node) {
            // the node's own post-collision populations, for the App. A terms:
            // float storage copies them to shared memory without holding
            // registers (waited for just before the lumps), half storage
            // loads them into registers
            static_for<1, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                if constexpr (G::CEN_SMEM)
                    cp_async4(cen_s + (unsigned)((A * G::threads + threadIdx.x) * 4),
                              fin + (plane_of<1, NS>(sp, A) * pstride + node));
                else
                    cen[A] = (float)fin[plane_of<1, NS>(sp, A) * pstride + node];
            });
            if constexpr (G::LOCAL) cenr = (float)fin[ref_plane<1, NS>(sp) * pstride + node];
        }
        const bool ok = mbar_wait_bounded(full(slot), (unsigned)((idx / SLOTS) & 1), wait_polls);
        // half storage: this stage's node densities around the node (the
        // density term of every stencil is taken from them once per stage)
        float rd[3][3] = {};
        if constexpr (G::LOCAL)
            if (ok) dens_block<NS, S, TY, SLOTS>(base, sp, tx, ty, rd);
        if (ok && unit_fast) {
            static_for<0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                constexpr int ez = ev<1>(A, 2);
                const float dI = rd[1 - ev<1>(A, 1)][1 - ev<1>(A, 0)], wa = p.wl[wclass<1>(A)];
                if constexpr (ez == 0) {
                    f[A] = accN[A];
                    if (!halo) accN[A] = inplane_unit<A, NS, S, TY, SLOTS>(base, sp, tx, ty, dI, wa);
                } else if constexpr (ez > 0) {
                    // exact shift: node z takes slab z - 1, which arrived two iterations ago
                    f[A] = accA[A];
                    accA[A] = accB[A];
                    accB[A] = solid_slab ? 0.0f : inplane_unit<A, NS, S, TY, SLOTS>(base, sp, tx, ty, dI, wa);
                } else {
                    f[A] = solid_slab ? 0.0f : inplane_unit<A, NS, S, TY, SLOTS>(base, sp, tx, ty, dI, wa);
                }
            });
        } else if (ok) {
            float di[3][3] = {};   // [ey + 1][ex + 1]
            if constexpr (G::LOCAL)
                static_for<0, 9>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    di[K / 3][K % 3] = dens_interp<K % 3 - 1, K / 3 - 1>(rd, mx, my);
                });
            static_for<0, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                constexpr int ez = ev<1>(A, 2);
                const float dI = di[ev<1>(A, 1) + 1][ev<1>(A, 0) + 1], wa = p.wl[wclass<1>(A)];
                if constexpr (ez == 0) {
                    f[A] = accN[A];
                    if (!halo) accN[A] = inplane<A, NS, S, TY, SLOTS>(base, sp, tx, ty, mx, my, dI, wa);
                } else {
                    const float R =
                        solid_slab ? 0.0f : inplane<A, NS, S, TY, SLOTS>(base, sp, tx, ty, mx, my, dI, wa);
                    // slab k feeds the nodes at z = k+1 (oz=-1), k (0), k-1 (+1)
                    f[A] = accA[A] + w[widx(1, ez)] * R;
                    accA[A] = accB[A] + w[widx(0, ez)] * R;
                    accB[A] = w[widx(-1, ez)] * R;
                }
            });
        }

        // ---- node (x, y, zo): wall terms, correction, moments
        float rho = 1.0f, drho = 0.0f, ueq[3] = {0.0f, 0.0f, 0.0f};
        if (ok && emit) {
            if (wall_node) {
                if constexpr (G::CEN_SMEM) cp_async_wait_all();
                const float* cs = reinterpret_cast<const float*>(smem + G::cen_offset) + threadIdx.x;
                const float4* L = lumps + ((wcls_xy + 9 * (zlo ? 1 : (zhi ? 2 : 0))) * NS + sp) * Q;
                static_for<1, Q>([&](auto ac) {
                    constexpr int A = decltype(ac)::value;
                    constexpr int AB = opp<1>(A);
                    const float4 l = __ldg(L + A);
                    if constexpr (G::LOCAL) {
                        const float wa = p.wl[wclass<1>(A)];
                        f[A] += l.x * fmaf(wa, cenr, cen[A]) + l.y * fmaf(wa, cenr, cen[AB]);
                    } else {   // deviations, plus the reference the weights carry
                        float ca, cb;
                        if constexpr (G::CEN_SMEM) { ca = cs[A * G::threads]; cb = cs[AB * G::threads]; }
                        else { ca = cen[A]; cb = cen[AB]; }
                        f[A] += l.x * ca + l.y * cb + p.ref[sp][wclass<1>(A)] * l.z;
                    }
                });
            }
            if (corr) {
                const float ci = (float)__ldg(corr + sp);
                static_for<0, Q>([&](auto ac) {
                    constexpr int A = decltype(ac)::value;
                    f[A] = fmaf(p.wl[wclass<1>(A)], ci, f[A]);
                });
            }
            // sums started from their first term (no explicit 0 + x)
            float r = f[0], j[3];
            static_for<1, Q>([&](auto ac) {
                constexpr int A = decltype(ac)::value;
                r += f[A];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    constexpr int first[3] = {first_dir<1>(0), first_dir<1>(1), first_dir<1>(2)};
                    const int e = ev<1>(A, d);
                    if (A == first[d]) j[d] = e > 0 ? f[A] : -f[A];
                    else if (e == 1) j[d] += f[A];
                    else if (e == -1) j[d] -= f[A];
                }
            });
            drho = r;
            if constexpr (Codec<S>::DARITH) r = p.rref[sp] + r;
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
        float rho_m = 0.0f, n = 0.0f;
#pragma unroll
        for (int i = 0; i < NS; ++i) { rho_m += r[i]; n += r[i] * p.Minv[i]; }
        const float rinv_m = __fdividef(1.0f, rho_m);
        float u[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < NS; ++i) acc += r[i] * ue[i][d];
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
        float V[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = 0.0f;
#pragma unroll
            for (int jj = 0; jj < NS; ++jj) {
                float xs = 0.0f;
#pragma unroll
                for (int i = 0; i < NS; ++i) xs = (i == sp) ? X[i][jj] : xs;
                if (jj != sp) acc += r[jj] * xs * (ueq[d] - ue[jj][d]);
            }
            V[d] = acc * rinv_m;
        }

        // ---- collision of this species (same algebra as the general kernel)
        const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const float ug = u[0] * p.g[0] + u[1] * p.g[1] + u[2] * p.g[2];
        float av[3], ua = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            av[d] = (ueq[d] - u[d]) * tau_inv - V[d];
            ua += u[d] * av[d];
        }
        constexpr bool DA = Codec<S>::DARITH;   // float: the deviation form of the general kernel
        const float Bc = tau_inv - inv_cs2 * ua;
        const float Bm = -inv_cs2 * ua;
        const float U2 = DA ? -0.5f * inv_cs2 * usq : 1.0f - 0.5f * inv_cs2 * usq;
        float dt[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (DA)
#pragma unroll
            for (int c = 0; c < 3; ++c) dt[c] = fmaf(p.wl[c], drho, p.refc[sp][c]);   // w rho - ref
        const float wr[3] = {p.wl[0] * rho, p.wl[1] * rho, p.wl[2] * rho};
        const float sr = rho * inv_cs2 * sfac;
        if (active) mass_acc += (double)rho;
        // half storage: the node density, rounded as stored, is the reference
        float rr = 0.0f;
        if constexpr (G::LOCAL) {
            rr = Codec<S>::rt(rho);
            if (active) Codec<S>::st(fout + (ref_plane<1, NS>(sp) * pstride + node), rr);
        }
        // Directions in opposite pairs (A, -A): with t1 = c e.u / c_s^2 and e.a,
        // e.g odd in e, each update is f + (even part) +- (odd part), the parts
        // formed once per pair.  Float (deviations):
        //   g* = g + (w rho - ref - g)/tau + w rho X + S,  X = phi (1/tau + b) + b,
        //   phi = t1 + t1^2/2 + U2, b = c/cs2 e.a + Bm, S = K (c e.g (1 + t1) - u.g);
        // half: f* = omt f + w rho (phi B) + S, B = c/cs2 e.a + Bc.
        const float cg[3] = {csp * p.g[0], csp * p.g[1], csp * p.g[2]};
        const float tB = DA ? tau_inv + Bm : Bc;
        auto emit_store = [&](int A, int C, float fs) {
            if (active) {
                if constexpr (G::LOCAL) Codec<S>::st(fout + (plane_of<1, NS>(sp, A) * pstride + node), fs - p.wl[C] * rr);
                else Codec<S>::st(fout + (plane_of<1, NS>(sp, A) * pstride + node), fs);
            }
        };
        static_for<0, Q>([&](auto ac) {
            constexpr int A = decltype(ac)::value;
            constexpr int AB = opp<1>(A);
            constexpr int C = wclass<1>(A);
            const float K = p.wl[C] * sr;
            if constexpr (A == 0) {
                // rest: t1 = e.a = e.g = 0
                const float S0 = -K * ug;
                float fs;
                if constexpr (DA) fs = f[0] + fmaf(tau_inv, dt[0] - f[0], fmaf(wr[0], fmaf(U2, tB, Bm), S0));
                else fs = fmaf(omt, f[0], fmaf(wr[0] * U2, Bc, S0));
                emit_store(0, 0, fs);
            } else if constexpr (A < AB) {
                const float t1 = c_inv_cs2 * edot<1, A>(u);
                const float bO = c_inv_cs2 * edot<1, A>(av);
                const float ceg = edot<1, A>(cg);
                const float phiE = fmaf(0.5f * t1, t1, U2);
                // even and odd parts of X (float) or of phi B (half)
                const float XE = DA ? fmaf(phiE, tB, fmaf(t1, bO, Bm)) : fmaf(phiE, tB, t1 * bO);
                const float XO = DA ? fmaf(t1, tB, fmaf(phiE, bO, bO)) : fmaf(t1, tB, phiE * bO);
                const float E = fmaf(wr[C], XE, K * fmaf(ceg, t1, -ug));
                const float O = fmaf(wr[C], XO, K * ceg);
                float fa, fb;
                if constexpr (DA) {   // g* directly: one large addition per direction
                    fa = f[A] + fmaf(tau_inv, dt[C] - f[A], E + O);
                    fb = f[AB] + fmaf(tau_inv, dt[C] - f[AB], E - O);
                } else {
                    fa = fmaf(omt, f[A], E + O);
                    fb = fmaf(omt, f[AB], E - O);
                }
                emit_store(A, C, fa);
                emit_store(AB, C, fb);
            }
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
        cp_async_wait_all();   // this thread's wall-population copies
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
    if (flags & F_MASS) {
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

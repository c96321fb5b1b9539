// lbve_kernels.cuh -- kernels of one time step of the coupled LB + Oldroyd-B method
// (Kuron et al., arXiv:2009.12279), templated on the PDF storage type.  Included by
// lbve_f64.cu (FP64 storage, FMA contraction off) and lbve_f32.cu (FP32/FP16/BF16
// storage with FP32 arithmetic), which instantiate them behind the launcher table of
// lbve_launch.h.
//
// Per step (split schedule):   k_momentum_exchange (links into tracked bodies)
//                              k_lb      : polymer force, moments, TRT collide, AA stream
//                              k_fv      : finite-volume stress update tau^t -> tau^{t+1}
// The fused schedule (k_fused) merges k_fv of step t with k_lb of step t+1.
#pragma once

#include <cstddef>
#include <type_traits>

#include "lbve_device.cuh"
#include "lbve_launch.h"

namespace lbve {

// 128-thread stream-collide blocks with a resident-block floor per SM, i.e. a register
// cap of 65536 / (128 x floor): without a cap the odd-parity kernel keeps all 37
// neighbour addresses live and drops to ~10 % occupancy.  Measured at 512^3: FP32 runs
// fastest at 7 blocks (72 registers; 8 blocks spill more, 9 or more lose); with the
// stochastically rounded 16-bit stores BF16 at 7 (4.00 ms against 4.03 at 8) and FP16 at
// 8 (4.03 ms against 4.09 at 7); FP64 keeps 8.
template <class S, int PAR>
constexpr int lb_min_blocks() {
    return (sizeof(S) == 4 || std::is_same<S, __nv_bfloat16>::value) ? 7 : 8;
}
// 256-thread stress blocks, 3 resident per SM (80 registers: no spills at 4)
#ifndef LBVE_FV_MIN_BLOCKS
#define LBVE_FV_MIN_BLOCKS 3
#endif
#ifndef LBVE_LBB_MIN_BLOCKS  // batched stream-collide (both parities in one kernel; the
#define LBVE_LBB_MIN_BLOCKS 7   // serving mix's pool step measured 1.201 ms at 7, 1.217 at 8)
#endif

template <class S>
struct KArgs {
    using R = typename Store<S>::R;
    Geo g;
    Phys<R> ph;
    S *f;
    const R *tau;     // stress at the time level read
    R *tau_out;       // stress at the next time level
    const R *u_in;    // velocity read by the stress update
    R *u_out;         // velocity written by the stream-collide
    const uint8_t *flag;
    const uint32_t *mask;
    const PartDev *parts;
    unsigned step;  // index of the step being performed (rounding keys of keyed stores)
    unsigned *bad;  // instability flag (mapped host word) or nullptr
    int zlo, zhi;   // planes the step kernels compute
    unsigned key_base;  // added to the cell index in rounding keys (a z-slab: its global offset)
    // per-direction / per-component bases (f + i np, tau + c np, u_out + k np, u_in + k np,
    // tau_out + c np), so that an address is one multiply-add of a 32-bit cell index; set
    // by link_dirs
    S *fq[Q];
    const R *tq[6];
    R *uq[3];
    const R *uiq[3];
    R *toq[6];
};

template <class S>
__host__ __device__ inline void link_dirs(KArgs<S> &a) {
    const size_t np = (size_t)a.g.np;
    for (int i = 0; i < Q; ++i) a.fq[i] = a.f + i * np;
    for (int c = 0; c < 6; ++c) a.tq[c] = a.tau + c * np;
    for (int k = 0; k < 3; ++k) a.uq[k] = a.u_out + k * np;
    for (int k = 0; k < 3; ++k) a.uiq[k] = a.u_in + k * np;
    for (int c = 0; c < 6; ++c) a.toq[c] = a.tau_out + c * np;
}

// Load f_i^t of cell r from its AA location for the given parity.
template <class S, int PAR>
__device__ __forceinline__ void load_pdfs(const KArgs<S> &a, const Cell &cl, unsigned r,
                                          typename Store<S>::R (&f)[Q]) {
    using R = typename Store<S>::R;
    const size_t np = (size_t)a.g.np;
    const R inv = a.ph.inv_scale;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S *p = PAR == 0 ? a.fq[i] + r : a.fq[copp(i)] + cl.idx(-cx(i), -cy(i), -cz(i));
        f[i] = Store<S>::ld(p, inv);
    }
}

// 6 w_i rho c_i . u_b of a link into a moving wall or particle cell (out of line: rare).
template <class R>
__device__ __noinline__ R moving_wall_term(const Geo &g, const Phys<R> &ph, const PartDev *parts, int fl, int xq,
                                           int yq, int zq, int i, R rho) {
    R ub[3];
    boundary_velocity<R>(g, ph, parts, fl, xq, yq, zq, ub);
    R cub = R(0);
    bool first = true;
    for (int k = 0; k < 3; ++k) {
        const int c = k == 0 ? cx(i) : (k == 1 ? cy(i) : cz(i));
        if (c != 0) {
            if (first) {
                cub = c > 0 ? ub[k] : -ub[k];
                first = false;
            } else {
                cub = c > 0 ? cub + ub[k] : cub - ub[k];
            }
        }
    }
    const R w = i < 7 ? wgt<R>(1) : wgt<R>(7);
    return R(6) * w * rho * cub;
}

// Store post-collision f*_i with AA addressing; links into solid cells bounce back with
// the moving-wall term of Eq. (ubb): f_-i(r, t+1) = f*_i(r) - 6 w_i rho c_i . u_b.
// Every f*_i also goes to its normal destination, unconditionally: when r + c_i is
// solid that slot belongs to the solid neighbour and is never read afterwards (even
// step: slot -i of r holds f_i(r + c_i)), or is the one this thread itself read before
// (odd step: slot i of r + c_i held the bounced population f_-i(r)).  The bounced value
// is an extra store for the links into solid cells only.
template <class S, int PAR>
__device__ __forceinline__ void store_pdfs(const KArgs<S> &a, const Cell &cl, unsigned r, uint32_t mask,
                                           const typename Store<S>::R (&fs)[Q], typename Store<S>::R rho) {
    using R = typename Store<S>::R;
    const size_t np = (size_t)a.g.np;
    const R sc = a.ph.scale;
    const bool moving = mask & MASK_MOVING;  // else every solid neighbour is a resting no-slip wall
    if constexpr (Store<S>::keyed) {
        // 16-bit storage: the pairs (i, -i) round together (stochastically, see Store); a
        // bounce from a resting wall stores the very bits of the normal store (one of the
        // two copies is never read), a moving-wall bounce rounds its own value
        const uint32_t h = fmix32((r + a.key_base) ^ (a.step * 0x9E3779B9u));
        const uint32_t d0 = Store<S>::round2(fs[0], fs[0], sc, pair_bits(h, 0));
        Store<S>::store16(a.fq[0] + r, d0);
        if (!__any_sync(__activemask(), moving)) {
            // no lane of the warp next to a moving boundary: every bounce is a predicated
            // store of the normal store's bits
#pragma unroll
            for (int i = 1; i < Q; i += 2) {
                const uint32_t d = Store<S>::round2(fs[i], fs[i + 1], sc, pair_bits(h, (i + 1) >> 1));
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = i + q;
                    const uint32_t bits = q == 0 ? d >> 16 : d;
                    const unsigned nb = cl.idx(cx(j), cy(j), cz(j));
                    Store<S>::store16(PAR == 0 ? a.fq[copp(j)] + r : a.fq[j] + nb, bits);
                    if (nb_solid(mask, j)) Store<S>::store16(PAR == 0 ? a.fq[j] + nb : a.fq[copp(j)] + r, bits);
                }
            }
            return;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const uint32_t d = Store<S>::round2(fs[i], fs[i + 1], sc, pair_bits(h, (i + 1) >> 1));
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = i + q;
                const uint32_t bits = q == 0 ? d >> 16 : d;
                const unsigned nb = cl.idx(cx(j), cy(j), cz(j));
                Store<S>::store16(PAR == 0 ? a.fq[copp(j)] + r : a.fq[j] + nb, bits);
                if (!nb_solid(mask, j)) continue;
                S *dst = PAR == 0 ? a.fq[j] + nb : a.fq[copp(j)] + r;
                const int fl = moving ? (int)a.flag[nb] : FLAG_NOSLIP;
                const R X = fl == FLAG_NOSLIP ? R(0)
                                              : moving_wall_term<R>(a.g, a.ph, a.parts, fl, cl.X(cx(j)), cl.Y(cy(j)),
                                                                    cl.Z(cz(j)), j, rho);
                // a boundary at rest (X exactly zero) bounces the normal store's bits
                Store<S>::store16(dst, X == R(0) ? bits
                                                 : Store<S>::round2(fs[j] - X, fs[j] - X, sc, pair_bits(h, Q + j)));
            }
        }
        return;
    }
    Store<S>::st(a.fq[0] + r, fs[0], sc);
    if (!__any_sync(__activemask(), moving)) {
        // no lane of the warp next to a moving boundary: bounce-back is a predicated store
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const unsigned nb = cl.idx(cx(i), cy(i), cz(i));
            Store<S>::st(PAR == 0 ? a.fq[copp(i)] + r : a.fq[i] + nb, fs[i], sc);
            if (nb_solid(mask, i)) Store<S>::st(PAR == 0 ? a.fq[i] + nb : a.fq[copp(i)] + r, fs[i], sc);
        }
        return;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const unsigned nb = cl.idx(cx(i), cy(i), cz(i));
        Store<S>::st(PAR == 0 ? a.fq[copp(i)] + r : a.fq[i] + nb, fs[i], sc);
        if (nb_solid(mask, i)) {
            R X = R(0);
            if (moving) {
                const int fl = a.flag[nb];
                if (fl != FLAG_NOSLIP)
                    X = moving_wall_term<R>(a.g, a.ph, a.parts, fl, cl.X(cx(i)), cl.Y(cy(i)), cl.Z(cz(i)), i, rho);
            }
            Store<S>::st(PAR == 0 ? a.fq[i] + nb : a.fq[copp(i)] + r, fs[i] - X, sc);
        }
    }
}

// LB half of the step for one fluid cell, given its own stress tr and an accessor tn for
// its face neighbours' stress (tau^t): F = g + F^p, moments, u^t written out, TRT
// collision with forcing, AA streaming with bounce-back.
template <class S, int PAR, bool FENE = false, class TauNb>
__device__ __forceinline__ void lb_core_f(const KArgs<S> &a, const Cell &cl, unsigned r, uint32_t mask,
                                          const typename Store<S>::R (&tr)[6], const TauNb &tn,
                                          typename Store<S>::R (&f)[Q]) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    R Fp[3], F[3], u[3], rho, drho;
    if constexpr (FENE)
        polymer_force_core_fene<R>(tr, mask, tn, a.ph, Fp);
    else
        polymer_force_core<R>(tr, mask, tn, Fp);
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = a.ph.g[k] + Fp[k];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    const size_t np = (size_t)a.g.np;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.uq[k][r] = u[k];
    const bool bad = collide<R, SH>(f, rho, drho, u, F, a.ph);
    store_pdfs<S, PAR>(a, cl, r, mask, f, rho);
    // instability (rho <= 0, |u| at or above the lattice sound speed, or a NaN): a rare
    // store to the host-mapped flag
    if (bad && a.bad != nullptr) *(volatile unsigned *)a.bad = 1u;
}
template <class S, int PAR, class TauNb>
__device__ __forceinline__ void lb_core(const KArgs<S> &a, const Cell &cl, unsigned r, uint32_t mask,
                                        const typename Store<S>::R (&tr)[6], const TauNb &tn) {
    typename Store<S>::R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    lb_core_f<S, PAR>(a, cl, r, mask, tr, tn, f);
}

// Velocity / stress / boundary-velocity accessors of the face neighbours in global memory.
template <class R>
struct GlobalNb {
    const Geo &g;
    const Phys<R> &ph;
    const Cell &cl;
    const R *tau;
    const R *u;
    const uint8_t *flag;
    const PartDev *parts;
    __device__ __forceinline__ unsigned at(int l) const {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        return cl.idx(k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0);
    }
    __device__ __forceinline__ R u_(int l, int j) const { return u[j * (size_t)g.np + at(l)]; }
    __device__ __forceinline__ R tau_(int l, int c) const { return tau[c * (size_t)g.np + at(l)]; }
    __device__ __forceinline__ void ub_(int l, R out[3]) const {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        const int dx = k == 0 ? s : 0, dy = k == 1 ? s : 0, dz = k == 2 ? s : 0;
        boundary_velocity_fast<R>(g, ph, parts, flag[at(l)], cl.X(dx), cl.Y(dy), cl.Z(dz), out);
    }
};
template <class R>
struct NbAdapter {  // gives GlobalNb the u / tau / ub interface fv_core expects
    const GlobalNb<R> &n;
    __device__ __forceinline__ R u(int l, int j) const { return n.u_(l, j); }
    __device__ __forceinline__ R tau(int l, int c) const { return n.tau_(l, c); }
    __device__ __forceinline__ void ub(int l, R out[3]) const { n.ub_(l, out); }
};

// Launch shape of the per-cell kernels: blockDim (bx, by), grid (nx/bx, ny/by, nz).
__device__ __forceinline__ bool cell_of_thread(const Geo &g, int &x, int &y, int &z) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z;
    return x < g.nx && y < g.ny;
}

// Stream-collide of the fluid cell (x, y, z) with the stress stencil read from global memory.
template <class S, int PAR, bool FENE = false>
__device__ __forceinline__ void lb_cell_at(const KArgs<S> &a, int x, int y, int z) {
    using R = typename Store<S>::R;
    const Cell cl(a.g, x, y, z);
    const unsigned r = cl.self();
    // the PDF and stress loads go out together with the mask (valid addresses for any
    // cell), not one DRAM round trip after it
    R f[Q], tr[6];
    load_pdfs<S, PAR>(a, cl, r, f);
#pragma unroll
    for (int c = 0; c < 6; ++c) tr[c] = a.tq[c][r];
    const uint32_t m = a.mask[r];
    if (m & 1u) return;
    auto tn = [&](int l, int c) -> R {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        return a.tq[c][cl.idx(k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0)];
    };
    lb_core_f<S, PAR, FENE>(a, cl, r, m, tr, tn, f);
}

// FENE: the stress arrays hold FENE-P conformation tensors (see polymer_force_core_fene)
template <class S, int PAR, bool FENE = false>
__global__ void __launch_bounds__(128, lb_min_blocks<S, PAR>()) k_lb(KArgs<S> a) {
    int x, y, z;
    if (!cell_of_thread(a.g, x, y, z)) return;
    lb_cell_at<S, PAR, FENE>(a, x, y, z + a.zlo);
}

template <class S>
__global__ void __launch_bounds__(128) k_fv(KArgs<S> a) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    int x, y, z;
    if (!cell_of_thread(a.g, x, y, z)) return;
    const Cell cl(a.g, x, y, z);
    const unsigned r = cl.self();
    const size_t np = (size_t)a.g.np;
    const uint32_t m = a.mask[r];
    R out[6];
    if (m & 1u) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.tau_out[c * np + r] = R(0);
        return;
    }
    R tr[6], ur[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) tr[c] = a.tau[c * np + r];
#pragma unroll
    for (int j = 0; j < 3; ++j) ur[j] = a.u_in[j * np + r];
    const GlobalNb<R> gn{a.g, a.ph, cl, a.tau, a.u_in, a.flag, a.parts};
    const NbAdapter<R> nb{gn};
    fv_core<R, SH, true>(a.ph, tr, ur, m, nb, out);
#pragma unroll
    for (int c = 0; c < 6; ++c) a.tau_out[c * np + r] = out[c];
}

// Neighbour masks of the cells in a box (whole grid: lo = 0, ext = n) from the flags.
// A neighbour outside a closed side counts as solid.
__device__ __forceinline__ uint32_t cell_mask(const Geo &g, const uint8_t *__restrict__ flag, int x, int y, int z) {
    const Cell cl(g, x, y, z);
    uint32_t m = flag[cl.self()] != FLAG_FLUID ? 1u : 0u;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const bool out = (!g.per[0] && (x + cx(i) < 0 || x + cx(i) >= g.nx)) ||
                         (!g.per[1] && (y + cy(i) < 0 || y + cy(i) >= g.ny)) ||
                         (!g.per[2] && (z + cz(i) < 0 || z + cz(i) >= g.nz));
        const int fl = out ? FLAG_NOSLIP : flag[cl.idx(cx(i), cy(i), cz(i))];
        if (fl != FLAG_FLUID) m |= 1u << i;
        if (fl != FLAG_FLUID && fl != FLAG_NOSLIP) m |= MASK_MOVING;
    }
    return m;
}

// Neighbour masks of the cells of a box (periodically wrapped); a non-fluid cell's stress
// is set to zero in both stress buffers, so that every solid cell holds zero stress (the
// shifted-mode stress update reads its face neighbours' stress without a solid test and
// selects a zero coefficient for a solid face).
template <class S>
__global__ void k_build_mask(Geo g, const uint8_t *__restrict__ flag, uint32_t *__restrict__ mask, int lx, int ly,
                             int lz, int ex, int ey, int ez, typename Store<S>::R *__restrict__ tau0,
                             typename Store<S>::R *__restrict__ tau1) {
    using R = typename Store<S>::R;
    const long long cells = (long long)ex * ey * ez;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cells;
         k += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(k % ex), iy = (int)((k / ex) % ey), iz = (int)(k / ((long long)ex * ey));
        const int x = ((lx + ix) % g.nx + g.nx) % g.nx;
        const int y = ((ly + iy) % g.ny + g.ny) % g.ny;
        const int z = ((lz + iz) % g.nz + g.nz) % g.nz;
        const unsigned r = (unsigned)x + (unsigned)g.nx * ((unsigned)y + (unsigned)g.ny * (unsigned)z);
        const uint32_t m = cell_mask(g, flag, x, y, z);
        mask[r] = m;
        if (m & 1u) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                tau0[c * (size_t)g.np + r] = R(0);
                tau1[c * (size_t)g.np + r] = R(0);
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// fused schedule: one kernel per step t does the stress update of step t-1 (tau^t from
// tau^{t-1}, u^{t-1}) and the LB half of step t, marching along z through an x-y tile.
// tau^{t-1} and u^{t-1} planes are staged in shared memory with cp.async (two planes
// ahead), tau^t is kept for three planes so the polymer force of plane z reads its
// face neighbours from shared memory, and only the tile's own cells are written out.
// ---------------------------------------------------------------------------------
constexpr int FT_X = 32, FT_Y = 8;
constexpr int H2X = FT_X + 4, H2Y = FT_Y + 4, NH2 = H2X * H2Y;  // staged inputs
constexpr int H1X = FT_X + 2, H1Y = FT_Y + 2, NH1 = H1X * H1Y;  // tau^t and masks

template <class R>
struct FusedSmem {
    R in_tau[3][6][NH2];
    R in_u[3][3][NH2];
    R tnew[3][6][NH1];
    uint32_t mask[4][NH1];
};

struct FusedWork {
    int tiles_x, tiles_y, zchunk, nzchunks;
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class R>
__device__ __forceinline__ void cp_async_real(R *dst, const R *src) {
    if constexpr (sizeof(R) == 8)
        cp_async8(dst, src);
    else
        cp_async4(dst, src);
}
// Copy of one real that reads n (sizeof(R) or 0) bytes and zero-fills the rest: n = 0
// writes a zero without reading src (which must still be a valid address).
// 16-byte copy that reads n (16 or 0) bytes: both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, unsigned n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
template <class R>
__device__ __forceinline__ void cp_async_real_zfill(R *dst, const R *src, unsigned n) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(R) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
}

// wrapped coordinate along a side, or -1 outside a closed side
__device__ __forceinline__ int side_coord(int q, int n, int per) {
    if (q >= 0 && q < n) return q;
    if (!per) return -1;
    return ((q % n) + n) % n;
}

__device__ __forceinline__ int ring3(int z) { return ((z % 3) + 3) % 3; }
__device__ __forceinline__ int ring4(int z) { return ((z % 4) + 4) % 4; }

// Smem neighbour accessor of the fused stress update (the staged planes zz-1, zz, zz+1).
template <class S>
struct SmemNb {
    using R = typename Store<S>::R;
    const FusedSmem<R> &sm;
    const KArgs<S> &a;
    int sc, sd, su, c2, xg, yg, zg;
    __device__ __forceinline__ int slot(int l) const { return l == 4 ? su : (l == 5 ? sd : sc); }
    __device__ __forceinline__ int cell(int l) const {
        return l == 0 ? c2 + 1 : l == 1 ? c2 - 1 : l == 2 ? c2 + H2X : l == 3 ? c2 - H2X : c2;
    }
    __device__ __forceinline__ R u(int l, int j) const { return sm.in_u[slot(l)][j][cell(l)]; }
    __device__ __forceinline__ R tau(int l, int c) const { return sm.in_tau[slot(l)][c][cell(l)]; }
    __device__ __forceinline__ void ub(int l, R o[3]) const {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        int xq = xg + (k == 0 ? s : 0), yq = yg + (k == 1 ? s : 0), zq = zg + (k == 2 ? s : 0);
        xq = xq < 0 ? xq + a.g.nx : (xq >= a.g.nx ? xq - a.g.nx : xq);
        yq = yq < 0 ? yq + a.g.ny : (yq >= a.g.ny ? yq - a.g.ny : yq);
        zq = zq < 0 ? zq + a.g.nz : (zq >= a.g.nz ? zq - a.g.nz : zq);
        const int fl = a.flag[(unsigned)xq + (unsigned)a.g.nx * ((unsigned)yq + (unsigned)a.g.ny * (unsigned)zq)];
        boundary_velocity_fast<R>(a.g, a.ph, a.parts, fl, xq, yq, zq, o);
    }
};

template <class S, int PAR>
__global__ void __launch_bounds__(FT_X * FT_Y, sizeof(typename Store<S>::R) == 8 ? 1 : 3) k_fused(KArgs<S> a, FusedWork w) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    constexpr int NT = FT_X * FT_Y;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<R> &sm = *reinterpret_cast<FusedSmem<R> *>(smem_raw);
    const int tid = threadIdx.x;
    const int item = blockIdx.x;
    const int tx = item % w.tiles_x;
    const int ty = (item / w.tiles_x) % w.tiles_y;
    const int zc = item / (w.tiles_x * w.tiles_y);
    const int x0 = tx * FT_X, y0 = ty * FT_Y;
    const int z0 = zc * w.zchunk;
    const int z1 = min(a.g.nz, z0 + w.zchunk);
    const size_t np = (size_t)a.g.np;
    const unsigned nx = (unsigned)a.g.nx, nxy = (unsigned)a.g.nx * (unsigned)a.g.ny;

    // in-plane offsets of the cells this thread stages (H2: tid, tid + NT; H1: the same)
    // and of its own stress-update cells; -1 marks a cell outside a closed side
    int off2[2], off1[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int k2 = tid + q * NT;
        off2[q] = -1;
        if (k2 < NH2) {
            const int xg = side_coord(x0 - 2 + k2 % H2X, a.g.nx, a.g.per[0]);
            const int yg = side_coord(y0 - 2 + k2 / H2X, a.g.ny, a.g.per[1]);
            if (xg >= 0 && yg >= 0) off2[q] = xg + (int)nx * yg;
        }
        const int k1 = tid + q * NT;
        off1[q] = -1;
        if (k1 < NH1) {
            const int xg = side_coord(x0 - 1 + k1 % H1X, a.g.nx, a.g.per[0]);
            const int yg = side_coord(y0 - 1 + k1 / H1X, a.g.ny, a.g.per[1]);
            if (xg >= 0 && yg >= 0) off1[q] = xg + (int)nx * yg;
        }
    }

    // stage tau^{t-1}, u^{t-1} (H2 region) and neighbour masks (H1 region) of plane zz
    auto stage = [&](int zz) {
        const int zg = side_coord(zz, a.g.nz, a.g.per[2]);
        const int s3 = ring3(zz), s4 = ring4(zz);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k2 = tid + q * NT;
            if (k2 < NH2) {
                if (off2[q] < 0 || zg < 0) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) sm.in_tau[s3][c][k2] = R(0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) sm.in_u[s3][j][k2] = R(0);
                } else {
                    const unsigned r = (unsigned)off2[q] + nxy * (unsigned)zg;
#pragma unroll
                    for (int c = 0; c < 6; ++c) cp_async_real<R>(&sm.in_tau[s3][c][k2], a.tau + c * np + r);
#pragma unroll
                    for (int j = 0; j < 3; ++j) cp_async_real<R>(&sm.in_u[s3][j][k2], a.u_in + j * np + r);
                }
            }
            const int k1 = tid + q * NT;
            if (k1 < NH1) {
                if (off1[q] < 0 || zg < 0)
                    sm.mask[s4][k1] = 0xffffffffu;
                else
                    cp_async4(&sm.mask[s4][k1], a.mask + ((unsigned)off1[q] + nxy * (unsigned)zg));
            }
        }
        cp_async_commit();
    };

    const int ti = tid % FT_X, tj = tid / FT_X;
    const int x = x0 + ti, y = y0 + tj;
    const int kc = (ti + 1) + (tj + 1) * H1X;  // the thread's own cell in H1 coordinates
    const bool own_xy = x < a.g.nx && y < a.g.ny;

#pragma unroll 1
    for (int zz = z0 - 2; zz <= z0; ++zz) stage(zz);

    // plane zf: stress update tau^t (H1 region), then stream-collide of plane zf - 1
#pragma unroll 1
    for (int zf = z0 - 1; zf <= z1; ++zf) {
        cp_async_wait_all();
        __syncthreads();
        {
            const int sc = ring3(zf), sd = ring3(zf - 1), su = ring3(zf + 1), s4 = ring4(zf);
            const int zg = side_coord(zf, a.g.nz, a.g.per[2]);
            const bool own_plane = zf >= z0 && zf < z1;
#pragma unroll 1
            for (int k = tid; k < NH1; k += NT) {
                const int hi = k % H1X, hj = k / H1X;
                const uint32_t m = sm.mask[s4][k];
                R out[6];
                if (m & 1u) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) out[c] = R(0);
                } else {
                    const int c2 = (hi + 1) + (hj + 1) * H2X;
                    R tr[6], ur[3];
#pragma unroll
                    for (int c = 0; c < 6; ++c) tr[c] = sm.in_tau[sc][c][c2];
#pragma unroll
                    for (int j = 0; j < 3; ++j) ur[j] = sm.in_u[sc][j][c2];
                    const int xg = side_coord(x0 - 1 + hi, a.g.nx, a.g.per[0]);
                    const int yg = side_coord(y0 - 1 + hj, a.g.ny, a.g.per[1]);
                    const SmemNb<S> nb{sm, a, sc, sd, su, c2, xg, yg, zg};
                    fv_core<R, SH, true>(a.ph, tr, ur, m, nb, out);
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) sm.tnew[sc][c][k] = out[c];
                if (own_plane && hi >= 1 && hi <= FT_X && hj >= 1 && hj <= FT_Y) {
                    const int xo = x0 + hi - 1, yo = y0 + hj - 1;
                    if (xo < a.g.nx && yo < a.g.ny) {
                        const unsigned r = (unsigned)xo + nx * (unsigned)yo + nxy * (unsigned)zf;
#pragma unroll
                        for (int c = 0; c < 6; ++c) a.tau_out[c * np + r] = out[c];
                    }
                }
            }
        }
        __syncthreads();
        if (zf + 2 <= z1 + 1) stage(zf + 2);
        const int z = zf - 1;
        if (z >= z0 && own_xy) {
            const uint32_t m = sm.mask[ring4(z)][kc];
            if (!(m & 1u)) {
                const int sc = ring3(z), sd = ring3(z - 1), su = ring3(z + 1);
                R tr[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) tr[c] = sm.tnew[sc][c][kc];
                auto tn = [&](int l, int c) -> R {
                    const int slot = l == 4 ? su : (l == 5 ? sd : sc);
                    const int cell = l == 0 ? kc + 1 : l == 1 ? kc - 1 : l == 2 ? kc + H1X : l == 3 ? kc - H1X : kc;
                    return sm.tnew[slot][c][cell];
                };
                const Cell cl(a.g, x, y, z);
                lb_core<S, PAR>(a, cl, cl.self(), m, tr, tn);
            }
        }
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------------
// stress update, z-marching: a block owns a 32 x 8 column of cells and walks a chunk of
// z-planes; tau^t and u^t of the planes z-1 .. z+2 (with a one-cell x-y halo) sit in a
// four-plane shared-memory ring filled with cp.async one plane ahead, so every stencil
// read of the update comes from shared memory.
// ---------------------------------------------------------------------------------
// Stress tiles: 256 threads over TX x (256 / TX) cells; the single-solve kernel uses
// 32 x 8, the batched kernel picks 16 x 16, 32 x 8 or 64 x 4 per solve.  A staged halo
// row holds the tile's TX cells from column XO on; W16 rows are widened to whole aligned
// 16-byte chunks (4 cells on each side) so that they are staged by 16-byte copies.
constexpr int FV_NT = 256;
constexpr int FV_X = 32, FV_Y = FV_NT / FV_X;
template <int TX, bool W16 = false>
struct FvTile {
    static constexpr int TY = FV_NT / TX;
    static constexpr int XO = W16 ? 4 : 1;
    static constexpr int HX = TX + 2 * XO, HN = HX * (TY + 2);  // halo row, halo cells
};
constexpr int FVH_X = FV_X + 2, FVH_Y = FV_Y + 2, FVH_N = FVH_X * FVH_Y;

// planes fetched beyond z + 1 while plane z is updated; the ring holds z - 1, z, z + 1
// and those
#ifndef LBVE_FV_AHEAD
#define LBVE_FV_AHEAD 1
#endif
constexpr int FV_RING = LBVE_FV_AHEAD + 3;
// ring slot of plane z (z >= -1); a power-of-two ring takes the low bits (two's complement)
__device__ __forceinline__ int fv_slot(int z) {
    if constexpr ((FV_RING & (FV_RING - 1)) == 0) return z & (FV_RING - 1);
    return ((z % FV_RING) + FV_RING) % FV_RING;
}

template <class R, int NH = FVH_N>
struct FvSmem {
    R tau[FV_RING][6][NH];
    R u[FV_RING][3][NH];
};

template <class S, int HX, int NH>
struct FvSmemNb {
    using R = typename Store<S>::R;
    const FvSmem<R, NH> &sm;
    const KArgs<S> &a;
    int sc, sd, su, c, xg, yg, zg;
    __device__ __forceinline__ int slot(int l) const { return l == 4 ? su : (l == 5 ? sd : sc); }
    __device__ __forceinline__ int cell(int l) const {
        return l == 0 ? c + 1 : l == 1 ? c - 1 : l == 2 ? c + HX : l == 3 ? c - HX : c;
    }
    __device__ __forceinline__ R u(int l, int j) const { return sm.u[slot(l)][j][cell(l)]; }
    __device__ __forceinline__ R tau(int l, int cc) const { return sm.tau[slot(l)][cc][cell(l)]; }
    __device__ __forceinline__ void ub(int l, R o[3]) const {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        int xq = xg + (k == 0 ? s : 0), yq = yg + (k == 1 ? s : 0), zq = zg + (k == 2 ? s : 0);
        xq = xq < 0 ? xq + a.g.nx : (xq >= a.g.nx ? xq - a.g.nx : xq);
        yq = yq < 0 ? yq + a.g.ny : (yq >= a.g.ny ? yq - a.g.ny : yq);
        zq = zq < 0 ? zq + a.g.nz : (zq >= a.g.nz ? zq - a.g.nz : zq);
        const int fl = a.flag[(unsigned)xq + (unsigned)a.g.nx * ((unsigned)yq + (unsigned)a.g.ny * (unsigned)zq)];
        boundary_velocity_fast<R>(a.g, a.ph, a.parts, fl, xq, yq, zq, o);
    }
};

// Stress update of work item `item` (TX x TY tile, z-chunk) of one solve; VAR compiles in
// the optional finite-volume variants, ZR the restriction to planes [zlo, zhi) of a
// z-slab (a separate build: the plain one keeps its register budget).  W16 stages the
// planes by 16-byte copies: 4-byte reals, nx a multiple of 4 and 16-byte aligned stress
// and velocity arrays (the launcher checks); the result is the same either way.  PB:
// the arguments are kernel parameters, so the per-component bases (tq, uiq, toq) are
// operands for free; the batched kernel (arguments in shared memory) forms base + c np.
template <class S, int TX, bool VAR, bool ZR = false, bool W16 = false, bool PB = false>
__device__ __forceinline__ void fv_tile(const KArgs<S> &a, FvSmem<typename Store<S>::R, FvTile<TX, W16>::HN> &sm,
                                        int item, int zchunk) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    using T = FvTile<TX, W16>;
    constexpr int NT = FV_NT, TY = T::TY, FVH_X = T::HX, FVH_N = T::HN, XO = T::XO;
    static_assert(!W16 || sizeof(R) == 4, "16-byte staging of 4-byte reals");
    static_assert(FVH_N <= 2 * NT, "two halo cells per thread at most");
    const int tid = threadIdx.x;
    const int tiles_x = (a.g.nx + TX - 1) / TX, tiles_y = (a.g.ny + TY - 1) / TY;
    const int tx = item % tiles_x, ty = (item / tiles_x) % tiles_y, zc = item / (tiles_x * tiles_y);
    const int x0 = tx * TX, y0 = ty * TY;
    const int z0 = ZR ? a.zlo + zc * zchunk : zc * zchunk;
    const int z1 = ZR ? min(a.zhi, z0 + zchunk) : min(a.g.nz, z0 + zchunk);
    const size_t np = (size_t)a.g.np;
    const unsigned nx = (unsigned)a.g.nx, nxy = (unsigned)a.g.nx * (unsigned)a.g.ny;
    auto tau_in = [&](int c) -> const R * {
        if constexpr (PB) return a.tq[c];
        return a.tau + c * np;
    };
    auto u_in = [&](int j) -> const R * {
        if constexpr (PB) return a.uiq[j];
        return a.u_in + j * np;
    };
    auto tau_out = [&](int c) -> R * {
        if constexpr (PB) return a.toq[c];
        return a.tau_out + c * np;
    };
    // 4-byte staging: halo cells tid and tid + NT of each plane (plane offsets, -1 beyond
    // a closed side); 16-byte staging: one aligned 4-cell chunk of a halo row per thread
    // (threads below CH: stress components 0..4; CH .. 2 CH - 1: component 5 and u)
    constexpr int CPR = FVH_X / 4, CH = CPR * (TY + 2);
    static_assert(!W16 || 2 * CH <= NT, "two threads per 16-byte chunk position at most");
    int off[2] = {-1, -1};
    int dpos = 0;
    const int half = W16 ? tid / CH : 0;
    if constexpr (W16) {
        if (half < 2) {
            const int p = tid - half * CH, row = p / CPR, cq = p - row * CPR;
            dpos = row * FVH_X + 4 * cq;
            const int xg = side_coord(x0 - XO + 4 * cq, a.g.nx, a.g.per[0]);
            const int yg = side_coord(y0 - 1 + row, a.g.ny, a.g.per[1]);
            if (xg >= 0 && yg >= 0) off[0] = xg + (int)nx * yg;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = tid + q * NT;
            if (k < FVH_N) {
                const int xg = side_coord(x0 - 1 + k % FVH_X, a.g.nx, a.g.per[0]);
                const int yg = side_coord(y0 - 1 + k / FVH_X, a.g.ny, a.g.per[1]);
                if (xg >= 0 && yg >= 0) off[q] = xg + (int)nx * yg;
            }
        }
    }
    static_assert(W16 || FVH_N > NT, "the first halo cell of every thread exists");
    auto stage = [&](int zz) {
        const int zg = side_coord(zz, a.g.nz, a.g.per[2]);
        const int s4 = fv_slot(zz);
        if constexpr (W16) {
            if (half < 2) {
                const bool in = off[0] >= 0 && zg >= 0;
                const unsigned r = in ? (unsigned)off[0] + nxy * (unsigned)zg : 0u;
                const unsigned n = in ? 16u : 0u;
                if (half == 0) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) cp_async16_zfill(&sm.tau[s4][c][dpos], tau_in(c) + r, n);
                } else {
                    cp_async16_zfill(&sm.tau[s4][5][dpos], tau_in(5) + r, n);
#pragma unroll
                    for (int j = 0; j < 3; ++j) cp_async16_zfill(&sm.u[s4][j][dpos], u_in(j) + r, n);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = tid + q * NT;
                if (q > 0 && k >= FVH_N) continue;
                // a halo cell beyond a closed side is zero-filled by the copy itself
                const bool in = off[q] >= 0 && zg >= 0;
                const unsigned r = in ? (unsigned)off[q] + nxy * (unsigned)zg : 0u;
                const unsigned n = in ? (unsigned)sizeof(R) : 0u;
#pragma unroll
                for (int c = 0; c < 6; ++c) cp_async_real_zfill<R>(&sm.tau[s4][c][k], tau_in(c) + r, n);
#pragma unroll
                for (int j = 0; j < 3; ++j) cp_async_real_zfill<R>(&sm.u[s4][j][k], u_in(j) + r, n);
            }
        }
        cp_async_commit();
    };
    const int ti = tid % TX, tj = tid / TX;
    const int x = x0 + ti, y = y0 + tj;
    const int kc = (ti + XO) + (tj + 1) * FVH_X;
    const bool own = x < a.g.nx && y < a.g.ny;
#pragma unroll
    for (int q = -1; q <= LBVE_FV_AHEAD; ++q) stage(z0 + q);
    // the mask of the next plane is fetched one plane ahead
    uint32_t m_next = own ? a.mask[(unsigned)x + nx * (unsigned)y + nxy * (unsigned)z0] : 1u;
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        const uint32_t m = m_next;
        if (own && z + 1 < z1) m_next = a.mask[(unsigned)x + nx * (unsigned)y + nxy * (unsigned)(z + 1)];
        // plane z + 1 + AHEAD is fetched while plane z is updated (an empty group keeps
        // the count); it goes to the slot of plane z - 2, free since the barrier that
        // ended the previous plane; planes up to z + 1 have landed
        if (z + 1 + LBVE_FV_AHEAD <= z1)
            stage(z + 1 + LBVE_FV_AHEAD);
        else
            cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(LBVE_FV_AHEAD) : "memory");
        __syncthreads();
        if (own) {
            const unsigned r = (unsigned)x + nx * (unsigned)y + nxy * (unsigned)z;
            R out[6];
            if (m & 1u) {
#pragma unroll
                for (int c = 0; c < 6; ++c) out[c] = R(0);
            } else {
                const int sc = fv_slot(z), sd = fv_slot(z - 1), su = fv_slot(z + 1);
                R tr[6], ur[3];
#pragma unroll
                for (int c = 0; c < 6; ++c) tr[c] = sm.tau[sc][c][kc];
#pragma unroll
                for (int j = 0; j < 3; ++j) ur[j] = sm.u[sc][j][kc];
                const FvSmemNb<S, FVH_X, FVH_N> nb{sm, a, sc, sd, su, kc, x, y, z};
                fv_core<R, SH, VAR>(a.ph, tr, ur, m, nb, out);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) tau_out(c)[r] = out[c];
        }
        __syncthreads();  // the next stage overwrites the slot of plane z - 1
    }
    cp_async_wait_all();
}

template <class S, bool VAR, bool ZR = false, bool W16 = false>
__global__ void __launch_bounds__(FV_X * FV_Y, sizeof(typename Store<S>::R) == 8 ? 2 : LBVE_FV_MIN_BLOCKS) k_fv_tiled(KArgs<S> a, int zchunk) {
    using R = typename Store<S>::R;
    extern __shared__ __align__(16) unsigned char fv_smem_raw[];
    using Sm = FvSmem<R, FvTile<FV_X, W16>::HN>;
    Sm &sm = *reinterpret_cast<Sm *>(fv_smem_raw);
    fv_tile<S, FV_X, VAR, ZR, W16, true>(a, sm, blockIdx.x, zchunk);
}

// ---------------------------------------------------------------------------------
// Two-cell stress update (the shifted modes' plain build: flux and source on, no
// variant).  As k_fv_tiled, a block marches a column through a z-chunk with the tau and u
// planes (one-cell halo in y, four cells in x: whole 16-byte chunks) staged in a
// four-plane shared-memory ring one plane ahead; the column is 64 x 8 cells and each of
// the 256 threads updates the cells x, x + 1 of one row in the two lanes of fv_core_sh
// (paired FP32 instructions), so the results are bitwise those of k_fv_tiled.
// ---------------------------------------------------------------------------------
constexpr int FP_TX = 64, FP_TY = 8, FP_NT = 256;
constexpr int FP_XO = 4, FP_HX = FP_TX + 2 * FP_XO, FP_HY = FP_TY + 2, FP_HN = FP_HX * FP_HY;
constexpr int FP_CPR = FP_HX / 4, FP_CH = FP_CPR * FP_HY;  // 16-byte chunks per halo row, per plane
struct FvPairSmem {
    float tau[FV_RING][6][FP_HN];
    float u[FV_RING][3][FP_HN];
};

template <class S, bool ZR>
__global__ void __launch_bounds__(FP_NT, 2) k_fv_pair(KArgs<S> a, int zchunk) {
    static_assert(Store<S>::shifted, "two-cell stress update: FP32 stress");
    extern __shared__ __align__(16) unsigned char fp_smem_raw[];
    FvPairSmem &sm = *reinterpret_cast<FvPairSmem *>(fp_smem_raw);
    const int tid = threadIdx.x;
    const int nx = a.g.nx, ny = a.g.ny;
    const int tiles_x = (nx + FP_TX - 1) / FP_TX, tiles_y = (ny + FP_TY - 1) / FP_TY;
    const int item = blockIdx.x;
    const int tx = item % tiles_x, ty = (item / tiles_x) % tiles_y, zc = item / (tiles_x * tiles_y);
    const int x0 = tx * FP_TX, y0 = ty * FP_TY;
    const int z0 = ZR ? a.zlo + zc * zchunk : zc * zchunk;
    const int z1 = ZR ? min(a.zhi, z0 + zchunk) : min(a.g.nz, z0 + zchunk);
    const unsigned nxu = (unsigned)nx, nxy = (unsigned)nx * (unsigned)ny;
    // staging: chunk positions tid and tid + FP_NT of 2 FP_CH (the first FP_CH carry tau
    // components 0..4, the others component 5 and u); -1 beyond a closed side
    int off[2], dpos[2], half[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int p = tid + q * FP_NT;
        half[q] = p < 2 * FP_CH ? p / FP_CH : 2;
        off[q] = -1;
        dpos[q] = 0;
        if (half[q] < 2) {
            const int pp = p - half[q] * FP_CH, row = pp / FP_CPR, cq = pp - row * FP_CPR;
            dpos[q] = row * FP_HX + 4 * cq;
            const int xg = side_coord(x0 - FP_XO + 4 * cq, nx, a.g.per[0]);
            const int yg = side_coord(y0 - 1 + row, ny, a.g.per[1]);
            if (xg >= 0 && yg >= 0) off[q] = xg + nx * yg;
        }
    }
    auto stage = [&](int zz) {
        const int zg = side_coord(zz, a.g.nz, a.g.per[2]);
        const int s4 = fv_slot(zz);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (half[q] >= 2) continue;
            const bool in = off[q] >= 0 && zg >= 0;
            const unsigned r = in ? (unsigned)off[q] + nxy * (unsigned)zg : 0u;
            const unsigned n = in ? 16u : 0u;
            if (half[q] == 0) {
#pragma unroll
                for (int c = 0; c < 5; ++c) cp_async16_zfill(&sm.tau[s4][c][dpos[q]], a.tq[c] + r, n);
            } else {
                cp_async16_zfill(&sm.tau[s4][5][dpos[q]], a.tq[5] + r, n);
#pragma unroll
                for (int j = 0; j < 3; ++j) cp_async16_zfill(&sm.u[s4][j][dpos[q]], a.uiq[j] + r, n);
            }
        }
        cp_async_commit();
    };
    const int ti = tid % (FP_TX / 2), tj = tid / (FP_TX / 2);
    const int x = x0 + 2 * ti, y = y0 + tj;
    const int kc = (2 * ti + FP_XO) + (tj + 1) * FP_HX;
    const bool own = x < nx && y < ny;  // nx is a multiple of 4: x + 1 < nx too
#pragma unroll
    for (int q = -1; q <= LBVE_FV_AHEAD; ++q) stage(z0 + q);
    auto mask2 = [&](int zz) { return *reinterpret_cast<const uint2 *>(a.mask + ((unsigned)x + nxu * (unsigned)y + nxy * (unsigned)zz)); };
    uint2 m_next = own ? mask2(z0) : make_uint2(1u, 1u);
#pragma unroll 1
    for (int z = z0; z < z1; ++z) {
        const uint2 m = m_next;
        if (own && z + 1 < z1) m_next = mask2(z + 1);
        if (z + 1 + LBVE_FV_AHEAD <= z1)
            stage(z + 1 + LBVE_FV_AHEAD);
        else
            cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(LBVE_FV_AHEAD) : "memory");
        __syncthreads();
        if (own) {
            const unsigned r = (unsigned)x + nxu * (unsigned)y + nxy * (unsigned)z;
            const bool fa = !(m.x & 1u), fb = !(m.y & 1u);
            float2 out[6];
            if (fa || fb) {
                const int sc = fv_slot(z), sd = fv_slot(z - 1), su = fv_slot(z + 1);
                auto ld2 = [](const float *p) { return *reinterpret_cast<const float2 *>(p); };
                float2 tr[6], ur[3];
#pragma unroll
                for (int c = 0; c < 6; ++c) tr[c] = ld2(&sm.tau[sc][c][kc]);
#pragma unroll
                for (int j = 0; j < 3; ++j) ur[j] = ld2(&sm.u[sc][j][kc]);
                struct Nb {
                    const KArgs<S> &a;
                    const FvPairSmem &sm;
                    const float2 (&tr)[6];
                    const float2 (&ur)[3];
                    int sc, sd, su, kc, x, y, z;
                    __device__ __forceinline__ float2 val(const float (*pl)[FP_HN], int l, int q, float2 own2,
                                                          const float (*pd)[FP_HN], const float (*pu)[FP_HN]) const {
                        switch (l) {
                            case 0: return make_float2(own2.y, pl[q][kc + 2]);
                            case 1: return make_float2(pl[q][kc - 1], own2.x);
                            case 2: return *reinterpret_cast<const float2 *>(&pl[q][kc + FP_HX]);
                            case 3: return *reinterpret_cast<const float2 *>(&pl[q][kc - FP_HX]);
                            case 4: return *reinterpret_cast<const float2 *>(&pu[q][kc]);
                            default: return *reinterpret_cast<const float2 *>(&pd[q][kc]);
                        }
                    }
                    __device__ __forceinline__ float2 u(int l, int k) const {
                        return val(sm.u[sc], l, k, ur[k], sm.u[sd], sm.u[su]);
                    }
                    __device__ __forceinline__ float2 tau(int l, int c) const {
                        return val(sm.tau[sc], l, c, tr[c], sm.tau[sd], sm.tau[su]);
                    }
                    __device__ __forceinline__ void ub(int l, int ln, float o[3]) const {
                        const int kk = l >> 1, sg = (l & 1) ? -1 : 1;
                        int xq = x + ln + (kk == 0 ? sg : 0), yq = y + (kk == 1 ? sg : 0), zq = z + (kk == 2 ? sg : 0);
                        xq = xq < 0 ? xq + a.g.nx : (xq >= a.g.nx ? xq - a.g.nx : xq);
                        yq = yq < 0 ? yq + a.g.ny : (yq >= a.g.ny ? yq - a.g.ny : yq);
                        zq = zq < 0 ? zq + a.g.nz : (zq >= a.g.nz ? zq - a.g.nz : zq);
                        const int fl = a.flag[(unsigned)xq +
                                              (unsigned)a.g.nx * ((unsigned)yq + (unsigned)a.g.ny * (unsigned)zq)];
                        boundary_velocity_fast<float>(a.g, a.ph, a.parts, fl, xq, yq, zq, o);
                    }
                };
                const Nb nb{a, sm, tr, ur, sc, sd, su, kc, x, y, z};
                fv_core_sh<float2, uint2, false>(a.ph, tr, ur, m, nb, out);
#pragma unroll
                for (int c = 0; c < 6; ++c) out[c] = make_float2(fa ? out[c].x : 0.0f, fb ? out[c].y : 0.0f);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) out[c] = make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) *reinterpret_cast<float2 *>(a.toq[c] + r) = out[c];
        }
        __syncthreads();  // the next stage overwrites the slot of plane z - 1
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------------
// batched schedule: the resident solves of a pool advance together.  Each kernel is a
// persistent grid over a packed list of work items (solve, block); a block reads the
// solve's descriptor into shared memory and runs the same per-cell code as the
// single-solve kernels, so every cell's arithmetic is the same alone and in the mix.
// ---------------------------------------------------------------------------------
constexpr int BLB_X = 32, BLB_Y = 4;  // cells per stream-collide work item

template <class S>
struct BatchEntry {
    KArgs<S> a[2];   // arguments for even / odd steps k of a launch sequence (k odd swaps
                     // the stress / velocity ping-pong), pointers linked on the host
    int parity0;     // AA parity at k = 0
    int lb_first, lb_items;
    int fv_first, fv_items, fv_zchunk;
    int lb_tx;       // stream-collide tile: lb_tx x (128 / lb_tx) cells (16, 32, 64, 128)
    int fv_tx;       // stress tile: fv_tx x (256 / fv_tx) cells (16, 32, 64; 32 for FP64)
};

// Stress tile widths the batched kernels support for real type R (FP64: 32 x 8 only,
// which keeps 2 blocks per SM).
template <class R>
struct FvBatchTiles {
    static constexpr bool wide = sizeof(R) == 4;
    __host__ __device__ static bool ok(int tx) { return tx == 32 || (wide && (tx == 16 || tx == 64)); }
};

// the entry whose [first, first + items) range holds work item `it` (binary search)
template <class S>
__device__ __forceinline__ int batch_find(const BatchEntry<S> *__restrict__ e, int n, int it, bool fv) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int first = fv ? e[mid].fv_first : e[mid].lb_first;
        if (first <= it)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Cooperative copy of a solve's arguments for step k into shared memory (all threads).
// The step index word gets `dstep` added: the steps the pool has taken since the
// arguments were built.
template <class S>
__device__ __forceinline__ void batch_load(KArgs<S> &sa, const BatchEntry<S> &e, int k, unsigned dstep, int tid,
                                           int nt) {
    static_assert(sizeof(KArgs<S>) % 4 == 0, "argument block copied as words");
    static_assert(offsetof(KArgs<S>, step) % 4 == 0, "step index is one word");
    constexpr int ws = (int)(offsetof(KArgs<S>, step) / 4);
    const unsigned *src = reinterpret_cast<const unsigned *>(&e.a[k & 1]);
    unsigned *dst = reinterpret_cast<unsigned *>(&sa);
    for (int w = tid; w < (int)(sizeof(KArgs<S>) / 4); w += nt) dst[w] = w == ws ? src[w] + dstep : src[w];
}

// Stream-collide over solves that all take AA parity PAR at this step (the pool keeps its
// members in two lists by parity and launches one kernel per list and step).
template <class S, int PAR>
__global__ void __launch_bounds__(BLB_X * BLB_Y, LBVE_LBB_MIN_BLOCKS) k_lb_batched(const BatchEntry<S> *__restrict__ e,
                                                                                 int nsolves, int total, int k,
                                                                                 const unsigned *__restrict__ dstep) {
    __shared__ KArgs<S> sa;
    const int tid = threadIdx.x;  // 1-D blocks of BLB_X * BLB_Y threads
    // items blockIdx.x, + gridDim.x, ...: the resident blocks sweep neighbouring tiles
    // together (halos shared through L2); a block's items only increase, so its solve
    // advances by a forward scan
    if ((int)blockIdx.x >= total) return;
    const unsigned ds = *dstep;
    int sv = batch_find<S>(e, nsolves, blockIdx.x, false), end = -1, first = 0, lx = 5;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        if (it >= end) {
            while (it >= e[sv].lb_first + e[sv].lb_items) ++sv;
            first = e[sv].lb_first;
            end = first + e[sv].lb_items;
            lx = __ffs(e[sv].lb_tx) - 1;  // log2 of the tile width
            __syncthreads();  // every thread is done with the previous solve's arguments
            batch_load<S>(sa, e[sv], k, ds, tid, BLB_X * BLB_Y);
            __syncthreads();
        }
        const int local = it - first;
        const int tw = 1 << lx, th = (BLB_X * BLB_Y) >> lx;
        const int tiles_x = (sa.g.nx + tw - 1) >> lx, tiles_y = (sa.g.ny + th - 1) / th;
        const int bx = local % tiles_x, by = (local / tiles_x) % tiles_y, z = local / (tiles_x * tiles_y);
        const int x = (bx << lx) + (tid & (tw - 1)), y = by * th + (tid >> lx);
        if (x < sa.g.nx && y < sa.g.ny) lb_cell_at<S, PAR>(sa, x, y, z);
    }
}

// Batched stress update over the solves whose stress tile is TX wide (the pool launches
// one of these per tile width present; fv_first counts within that group).  VAR when a
// solve of the group uses a finite-volume variant (the others compute as without it).
template <class S, int TX, bool VAR>
__global__ void __launch_bounds__(FV_NT, sizeof(typename Store<S>::R) == 8 ? 2 : LBVE_FV_MIN_BLOCKS) k_fv_batched(
    const BatchEntry<S> *__restrict__ e, int nsolves, int total, int k) {
    using R = typename Store<S>::R;
    extern __shared__ __align__(16) unsigned char fv_smem_raw[];
    FvSmem<R, FvTile<TX>::HN> &sm = *reinterpret_cast<FvSmem<R, FvTile<TX>::HN> *>(fv_smem_raw);
    __shared__ KArgs<S> sa;
    if ((int)blockIdx.x >= total) return;
    int sv = batch_find<S>(e, nsolves, blockIdx.x, true), end = -1, first = 0, zchunk = 1;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        if (it >= end) {
            while (it >= e[sv].fv_first + e[sv].fv_items) ++sv;
            first = e[sv].fv_first;
            end = first + e[sv].fv_items;
            zchunk = e[sv].fv_zchunk;
            __syncthreads();
            batch_load<S>(sa, e[sv], k, 0u, threadIdx.x, FV_NT);  // the stress update uses no step index
            __syncthreads();
        }
        fv_tile<S, TX, VAR>(sa, sm, it - first, zchunk);
        __syncthreads();
    }
}

// Residual of one solve: sums over fluid cells of |u - u_snap|^2 and |u|^2 (FP64,
// fixed-shape block partials), then u_snap = u.
template <class S>
__global__ void __launch_bounds__(256) k_residual(Geo g, const uint32_t *__restrict__ mask,
                                                  const typename Store<S>::R *__restrict__ u,
                                                  typename Store<S>::R *__restrict__ usnap, double *__restrict__ partial) {
    const size_t np = (size_t)g.np;
    double d2 = 0.0, u2 = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.n; r += (long long)gridDim.x * blockDim.x) {
        if (mask[r] & 1u) continue;
        for (int j = 0; j < 3; ++j) {
            const double v = (double)u[j * np + r], w = (double)usnap[j * np + r];
            d2 += (v - w) * (v - w);
            u2 += v * v;
            usnap[j * np + r] = u[j * np + r];
        }
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = d2;
    sh[1][threadIdx.x] = u2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sh[0][0];
        partial[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// ---------------------------------------------------------------------------------
// momentum exchange (Sec. "Moving boundaries"): for every link (fluid cell r,
// direction i into a tracked solid cell) the force c_i (2 f*_i - 6 w_i rho c_i.u_b) and
// its torque about the owning particle.  Runs before k_lb on the same f^t and repeats
// the cell's collision, so f*_i is exactly the value k_lb streams.
// ---------------------------------------------------------------------------------
// Momentum-exchange contribution of one link (code = r << 5 | i) into contrib[8].
template <class S, int PAR>
__device__ __forceinline__ void me_link(const KArgs<S> &a, long long code, double *__restrict__ o) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    const int i = (int)(code & 31);
    const unsigned r = (unsigned)(code >> 5);
    const int x = (int)(r % a.g.nx), y = (int)((r / a.g.nx) % a.g.ny), z = (int)(r / ((unsigned)a.g.nx * a.g.ny));
    const Cell cl(a.g, x, y, z);
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, a.ph, cl, r, a.mask[r], a.tau, Fp);
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = a.ph.g[k] + Fp[k];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    collide<R, SH>(f, rho, drho, u, F, a.ph);
    // f*_i (a full population: the stored deviation plus w_i rho0 in shifted modes)
    R fsi = R(0);
    int ci[3] = {0, 0, 0};
#pragma unroll
    for (int k = 1; k < Q; ++k)
        if (k == i) {
            fsi = f[k];
            ci[0] = cx(k);
            ci[1] = cy(k);
            ci[2] = cz(k);
        }
    const int xb = cl.X(ci[0]), yb = cl.Y(ci[1]), zb = cl.Z(ci[2]);
    const long long nb = (long long)xb + (long long)a.g.nx * (yb + (long long)a.g.ny * zb);
    const int fl = a.flag[nb];
    R ub[3];
    boundary_velocity<R>(a.g, a.ph, a.parts, fl, xb, yb, zb, ub);
    R cub = R(0);
    {
        bool first = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (ci[k] != 0) {
                if (first) {
                    cub = ci[k] > 0 ? ub[k] : -ub[k];
                    first = false;
                } else {
                    cub = ci[k] > 0 ? cub + ub[k] : cub - ub[k];
                }
            }
        }
    }
    const R wi = i < 7 ? wgt<R>(1) : wgt<R>(7);
    const R X = R(6) * wi * rho * cub;
    double m;
    if constexpr (SH)
        m = 2.0 * ((double)fsi + (double)(i < 7 ? wgt<double>(1) : wgt<double>(7)) * (double)a.ph.rho0) - (double)X;
    else
        m = 2.0 * fsi - X;
    const double Fl[3] = {ci[0] * m, ci[1] * m, ci[2] * m};
    double T[3] = {0.0, 0.0, 0.0};
    if (fl >= FLAG_PART0 && fl < FLAG_PART0 + MAX_PART) {
        const PartDev &P = a.parts[fl - FLAG_PART0];
        double q[3] = {(double)xb, (double)yb, (double)zb}, d[3];
        int nn[3] = {a.g.nx, a.g.ny, a.g.nz};
        for (int k = 0; k < 3; ++k) {
            d[k] = q[k] - P.X[k];
            if (a.g.per[k]) d[k] -= (double)nn[k] * floor(d[k] / (double)nn[k] + 0.5);
        }
        T[0] = d[1] * Fl[2] - d[2] * Fl[1];
        T[1] = d[2] * Fl[0] - d[0] * Fl[2];
        T[2] = d[0] * Fl[1] - d[1] * Fl[0];
    }
    o[0] = Fl[0];
    o[1] = Fl[1];
    o[2] = Fl[2];
    o[3] = T[0];
    o[4] = T[1];
    o[5] = T[2];
    o[6] = (double)fl;
}

// Momentum exchange over link segments (one segment per tracked body, blockIdx.y):
// link l of segment b is links[seg_begin[b] + l] for l < seg_count[b].
template <class S, int PAR>
__global__ void __launch_bounds__(128) k_momentum_exchange(KArgs<S> a, const long long *__restrict__ links,
                                                           const int *__restrict__ seg_begin,
                                                           const int *__restrict__ seg_count,
                                                           double *__restrict__ contrib) {
    const int b = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= seg_count[b]) return;
    const long long at = (long long)seg_begin[b] + l;
    me_link<S, PAR>(a, links[at], contrib + at * 8);
}

// Same with the links of a block summed inside the block (fixed tree order): one partial
// of 6 doubles (stride 8) per (body, block) at part[(b * gridDim.x + block) * 8].  The
// final per-body sum then reads ceil(count / 128) partials instead of every link.
template <class S, int PAR>
__global__ void __launch_bounds__(128) k_momentum_exchange_part(KArgs<S> a, const long long *__restrict__ links,
                                                                const int *__restrict__ seg_begin,
                                                                const int *__restrict__ seg_count,
                                                                double *__restrict__ part) {
    const int b = blockIdx.y;
    const int cnt = seg_count[b];
    if ((int)blockIdx.x * 128 >= cnt) return;  // the whole block is past this body's links
    const int l = blockIdx.x * 128 + threadIdx.x;
    double o[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (l < cnt) me_link<S, PAR>(a, links[(long long)seg_begin[b] + l], o);
    __shared__ double sh[6][128];
#pragma unroll
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = o[k];
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) part[((long long)b * gridDim.x + blockIdx.x) * 8 + k] = sh[k][0];
}

// ---------------------------------------------------------------------------------
// moving particles (Sec. "Moving boundaries")
// ---------------------------------------------------------------------------------
struct BBox {
    int lo[3], ext[3];
    __host__ __device__ long long cells() const { return (long long)ext[0] * ext[1] * ext[2]; }
};

// Cells within R + margin of the particle centre (whole domain along a periodic side
// the box would wrap onto itself; clamped to the domain along a closed side).
__host__ __device__ inline BBox particle_bbox(const Geo &g, const double X[3], double R, int margin) {
    BBox b;
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; ++k) {
        int lo = (int)floor(X[k] - R) - margin;
        int hi = (int)ceil(X[k] + R) + margin;
        if (!g.per[k]) {
            lo = lo < 0 ? 0 : lo;
            hi = hi > nn[k] - 1 ? nn[k] - 1 : hi;
        }
        int ext = hi - lo + 1;
        if (ext > nn[k]) {
            lo = 0;
            ext = nn[k];
        }
        if (ext < 0) ext = 0;
        b.lo[k] = lo;
        b.ext[k] = ext;
    }
    return b;
}

__host__ __device__ inline int bbox_capacity_side(double R, int margin) { return 2 * (int)ceil(R) + 2 * margin + 3; }

__device__ __forceinline__ int wrapc(int v, int n) { return ((v % n) + n) % n; }

__device__ __forceinline__ long long bbox_cell(const Geo &g, const BBox &b, long long k, int &x, int &y, int &z) {
    // a particle box holds far fewer than 2^32 cells: 32-bit division (64-bit division is
    // a long software sequence)
    const unsigned kk = (unsigned)k, row = kk / (unsigned)b.ext[0];
    const int ix = (int)(kk - row * (unsigned)b.ext[0]);
    const int iy = (int)(row % (unsigned)b.ext[1]);
    const int iz = (int)(row / (unsigned)b.ext[1]);
    x = wrapc(b.lo[0] + ix, g.nx);
    y = wrapc(b.lo[1] + iy, g.ny);
    z = wrapc(b.lo[2] + iz, g.nz);
    return (long long)x + (long long)g.nx * (y + (long long)g.ny * z);
}

// index of global cell (x, y, z) inside the box, or -1
__device__ __forceinline__ long long bbox_index(const Geo &g, const BBox &b, int x, int y, int z) {
    const int q[3] = {x, y, z}, nn[3] = {g.nx, g.ny, g.nz};
    int o[3];
    for (int k = 0; k < 3; ++k) {
        int d = q[k] - b.lo[k];
        if (g.per[k]) d = wrapc(d, nn[k]);
        if (d < 0 || d >= b.ext[k]) return -1;
        o[k] = d;
    }
    return (long long)o[0] + (long long)b.ext[0] * (o[1] + (long long)b.ext[1] * o[2]);
}

__device__ __forceinline__ void min_image(const Geo &g, const double X[3], int x, int y, int z, double d[3]) {
    const double q[3] = {(double)x, (double)y, (double)z};
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; ++k) {
        d[k] = q[k] - X[k];
        if (g.per[k]) d[k] -= (double)nn[k] * floor(d[k] / (double)nn[k] + 0.5);
    }
}

// Sphere test |r - X|^2 <= R^2 of Sec. "Moving boundaries" (minimum image), decided as in
// FP64 but mostly computed in FP32: FP64 runs at a small fraction of the FP32 rate here,
// and the fill/drain classification tests every cell of a particle's box each step.
// The FP32 distance differs from the FP64 one by less than `tol` (bounded from the
// magnitudes involved, see sphere_filter), so outside a shell |d^2 - R^2| <= tol the FP32
// outcome is the FP64 outcome; inside the shell the FP64 test decides.
struct SphereFilter {
    float X[3], inv_n[3], n[3], R2, tol;
};
__device__ __forceinline__ SphereFilter sphere_filter(const Geo &g, const PartDev &P) {
    SphereFilter f;
    const int nn[3] = {g.nx, g.ny, g.nz};
    double S = P.R + 4.0;
    for (int k = 0; k < 3; ++k) {
        f.X[k] = (float)P.X[k];
        f.n[k] = (float)nn[k];
        f.inv_n[k] = 1.0f / (float)nn[k];
        S += fabs(P.X[k]) + (double)nn[k];
    }
    f.R2 = (float)(P.R * P.R);
    // each FP32 displacement is within ~2^-21 S of the FP64 one (rounding of X, of the
    // difference and of the periodic shift); the sum of squares then within 2^-18 S^2, and
    // twice that is kept as the margin
    f.tol = (float)(S * S * 0x1p-17);
    return f;
}
__device__ __forceinline__ bool inside_sphere(const Geo &g, const PartDev &P, const SphereFilter &f, int x, int y,
                                              int z) {
    const int q[3] = {x, y, z};
    float d2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float dk = (float)q[k] - f.X[k];
        if (g.per[k]) dk -= f.n[k] * floorf(dk * f.inv_n[k] + 0.5f);
        d2 += dk * dk;
    }
    if (d2 < f.R2 - f.tol) return true;
    if (d2 > f.R2 + f.tol) return false;
    double d[3];
    min_image(g, P.X, x, y, z, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= P.R * P.R;
}

// Initial placement: covered fluid cells become particle cells, their stress is zeroed.
template <class S>
__global__ void k_voxelise(KArgs<S> a, PartDev *__restrict__ parts, int p, uint8_t *__restrict__ flag,
                           typename Store<S>::R *__restrict__ tau0, typename Store<S>::R *__restrict__ tau1) {
    using R = typename Store<S>::R;
    const PartDev &P = parts[p];
    const BBox b = particle_bbox(a.g, P.X, P.R, 1);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < b.cells(); k += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        const long long r = bbox_cell(a.g, b, k, x, y, z);
        if (flag[r] != FLAG_FLUID) continue;
        double d[3];
        min_image(a.g, P.X, x, y, z, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= P.R * P.R) {
            flag[r] = (uint8_t)(FLAG_PART0 + p);
            for (int c = 0; c < 6; ++c) {
                tau0[c * a.g.np + r] = R(0);
                tau1[c * a.g.np + r] = R(0);
            }
        }
    }
}

// Symplectic Euler (Sec. "Moving boundaries"): velocities with the momentum-exchange
// force and torque of this step plus the external ones, then the position with the new
// velocity.  One thread per particle, FP64.
__device__ __forceinline__ void particle_update_one(PartDev &P) {
    for (int k = 0; k < 3; ++k) {
        P.v[k] += (P.Fme[k] + P.Fext[k]) / P.m;
        P.w[k] += (P.Tme[k] + P.Text[k]) / P.I;
        P.X[k] += P.v[k];
    }
}
template <class S>
__global__ void k_particle_update(PartDev *__restrict__ parts, int nparts) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparts) return;
    particle_update_one(parts[p]);
}

// Boundary links of each particle (one block per particle): every (fluid cell r,
// direction i) with r + c_i covered by the particle, in cell order then direction
// order, compacted with a block-wide prefix sum so the order is deterministic.
template <class S, int NT>
__device__ __forceinline__ void particle_links_block(const Geo &g, const PartDev *__restrict__ parts, int p,
                                                     const uint8_t *__restrict__ flag, long long *__restrict__ links,
                                                     const int *__restrict__ seg_begin, int *__restrict__ seg_count,
                                                     int first_seg, const int *__restrict__ capacity) {
    const PartDev &P = parts[p];
    if (!P.changed) return;  // no cell converted since the last build: the links still hold
    const BBox b = particle_bbox(g, P.X, P.R, 2);
    const long long nc = b.cells();
    const int seg = first_seg + p;
    long long *out = links + seg_begin[seg];
    const int cap = capacity[p];
    constexpr int NW = NT / 32;
    __shared__ int wsum[NW];
    __shared__ int base;
    const int lane = (int)threadIdx.x & 31, warp = (int)threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (long long k0 = 0; k0 < nc; k0 += blockDim.x) {
        const long long k = k0 + threadIdx.x;
        unsigned mask = 0;
        long long r = 0;
        if (k < nc) {
            int x, y, z;
            r = bbox_cell(g, b, k, x, y, z);
            if (flag[r] == FLAG_FLUID) {
                const Cell cl(g, x, y, z);
                for (int i = 1; i < Q; ++i) {
                    if (!g.per[0] && (x + cx(i) < 0 || x + cx(i) >= g.nx)) continue;
                    if (!g.per[1] && (y + cy(i) < 0 || y + cy(i) >= g.ny)) continue;
                    if (!g.per[2] && (z + cz(i) < 0 || z + cz(i) >= g.nz)) continue;
                    if (flag[cl.idx(cx(i), cy(i), cz(i))] == FLAG_PART0 + p) mask |= 1u << i;
                }
            }
        }
        // warp-level compaction in thread order: a ballot skips warps without links, a
        // shuffle scan places each thread's links within its warp, the warp totals are
        // scanned by the first warp
        const int cnt = __popc(mask);
        int incl = 0;
        if (__ballot_sync(0xffffffffu, cnt != 0)) {
            incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t;
            }
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < NW ? wsum[lane] : 0;
#pragma unroll
            for (int off = 1; off < NW; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += t;
            }
            if (lane < NW) wsum[lane] = w;  // inclusive over the warps
        }
        __syncthreads();
        int pos = base + (warp ? wsum[warp - 1] : 0) + incl - cnt;
        for (int i = 1; i < Q; ++i)
            if (mask & (1u << i)) {
                if (pos < cap) out[pos] = (r << 5) | i;
                pos++;
            }
        __syncthreads();
        if (threadIdx.x == 0) base += wsum[NW - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) seg_count[seg] = base < cap ? base : cap;
}
template <class S>
__global__ void __launch_bounds__(256) k_particle_links(Geo g, const PartDev *__restrict__ parts,
                                                        const uint8_t *__restrict__ flag,
                                                        long long *__restrict__ links,
                                                        const int *__restrict__ seg_begin, int *__restrict__ seg_count,
                                                        int first_seg, const int *__restrict__ capacity) {
    particle_links_block<S, 256>(g, parts, (int)blockIdx.x, flag, links, seg_begin, seg_count, first_seg, capacity);
}

// Fill/drain after re-voxelisation at the particles' new positions (one block, the
// particles one after another).  f is the state at time t+1 in the layout PAR reads.
// kind: 0 other, 1 fluid before and after, 2 destroyed (fluid -> particle),
// 3 created (particle -> fluid).  All stress moves use the pre-conversion stress:
//   destroyed d: each of its N_f stable D3Q7 neighbours gains tau(d)/N_f;
//   created c:   tau(c) = sum of its stable neighbours' tau / (N_f + 1), each of
//                them gives up tau(c)/N_f;
// the deleted / created momentum goes to the particle as an impulse at the cell.
template <class S, int PAR>
__device__ __forceinline__ void fill_drain_block(const KArgs<S> &a, PartDev *__restrict__ parts, int nparts,
                                                 uint8_t *__restrict__ flag, uint32_t *__restrict__ mask,
                                                 typename Store<S>::R *__restrict__ tau,
                                                 uint8_t *__restrict__ kind, uint8_t *__restrict__ nf_arr,
                                                 double *__restrict__ delta, int *__restrict__ conv,
                                                 double *__restrict__ diag, double (*s_pm)[6]) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    const long long np = a.g.np;
    auto kind_of = [&](const BBox &b, int x, int y, int z) -> int {
        const long long k = bbox_index(a.g, b, x, y, z);
        if (k >= 0) return kind[k];
        return flag[(long long)x + (long long)a.g.nx * (y + (long long)a.g.ny * z)] == FLAG_FLUID ? 1 : 0;
    };
    for (int p = 0; p < nparts; ++p) {
        PartDev &P = parts[p];
        const BBox b = particle_bbox(a.g, P.X, P.R, 3);
        const long long nc = b.cells();
        const SphereFilter sf = sphere_filter(a.g, P);
        // A: classify (unrolled: several cells' flag loads in flight per thread)
        int any_local = 0;
#pragma unroll 4
        for (long long k = threadIdx.x; k < nc; k += blockDim.x) {
            int x, y, z;
            const long long r = bbox_cell(a.g, b, k, x, y, z);
            const int old = flag[r];
            int kd = 0;
            if (old == FLAG_FLUID || old == FLAG_PART0 + p) {
                const bool inside = inside_sphere(a.g, P, sf, x, y, z);
                if (old == FLAG_FLUID) kd = inside ? 2 : 1;
                else kd = inside ? 0 : 3;
            }
            kind[k] = (uint8_t)kd;
            any_local |= (kd == 2 || kd == 3);
        }
        if (!__syncthreads_or(any_local)) {
            // nothing converts: no impulse, flags and links stay as they are
            if (threadIdx.x == 0) {
                for (int c3 = 0; c3 < 3; ++c3) P.dP[c3] = P.dL[c3] = 0.0;
                P.changed = 0;
            }
            __syncthreads();
            continue;
        }
        // A': ordered list of the converted cells.  Each thread counts the converted cells
        // of its own contiguous range of the box, one block-wide exclusive scan of the
        // counts (warp shuffles, then the warp totals) gives each range's offset, and each
        // thread writes its cells in increasing order: the list is in cell order.
        __shared__ int s_wsum[32], s_total;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
        const long long per = (nc + blockDim.x - 1) / blockDim.x;
        const long long k_lo = min(nc, per * threadIdx.x), k_hi = min(nc, k_lo + per);
        int cnt = 0;
        for (long long k = k_lo; k < k_hi; ++k) cnt += (kind[k] == 2 || kind[k] == 3) ? 1 : 0;
        int incl = cnt;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int w = lane < nwarp ? s_wsum[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            if (lane < nwarp) s_wsum[lane] = wi - w;  // exclusive offsets of the warps
            if (lane == 31) s_total = wi;
        }
        __syncthreads();
        int pos = s_wsum[warp] + incl - cnt;
        for (long long k = k_lo; k < k_hi && pos < s_wsum[warp] + incl; ++k)
            if (kind[k] == 2 || kind[k] == 3) conv[pos++] = (int)k;
        const int nconv = s_total;
        __syncthreads();
        // B: N_f of converted cells, new stress of created cells
        for (int q = threadIdx.x; q < nconv; q += blockDim.x) {
            const long long k = conv[q];
            const int kd = kind[k];
            int x, y, z;
            bbox_cell(a.g, b, k, x, y, z);
            const Cell cl(a.g, x, y, z);
            int nf = 0;
            double sum[6] = {0, 0, 0, 0, 0, 0};
            for (int l = 0; l < 6; ++l) {
                const int ax = l >> 1, s = (l & 1) ? -1 : 1;
                const int xq = cl.X(ax == 0 ? s : 0), yq = cl.Y(ax == 1 ? s : 0), zq = cl.Z(ax == 2 ? s : 0);
                if (!a.g.per[ax]) {
                    const int q = ax == 0 ? x + s : (ax == 1 ? y + s : z + s);
                    const int nn = ax == 0 ? a.g.nx : (ax == 1 ? a.g.ny : a.g.nz);
                    if (q < 0 || q >= nn) continue;
                }
                if (kind_of(b, xq, yq, zq) != 1) continue;
                nf++;
                const long long nb = (long long)xq + (long long)a.g.nx * (yq + (long long)a.g.ny * zq);
                for (int c = 0; c < 6; ++c) sum[c] += (double)tau[c * np + nb];
            }
            nf_arr[k] = (uint8_t)nf;
            if (kd == 3)
                for (int c = 0; c < 6; ++c) delta[c * nc + k] = sum[c] / (double)(nf + 1);
        }
        __syncthreads();
        // C: stress gathered by each stable cell from its converted D3Q7 neighbours
        for (long long k = threadIdx.x; k < nc; k += blockDim.x) {
            if (kind[k] != 1) continue;
            int x, y, z;
            bbox_cell(a.g, b, k, x, y, z);
            const Cell cl(a.g, x, y, z);
            double acc[6] = {0, 0, 0, 0, 0, 0};
            bool touched = false;
            for (int l = 0; l < 6; ++l) {
                const int ax = l >> 1, s = (l & 1) ? -1 : 1;
                if (!a.g.per[ax]) {
                    const int q = ax == 0 ? x + s : (ax == 1 ? y + s : z + s);
                    const int nn = ax == 0 ? a.g.nx : (ax == 1 ? a.g.ny : a.g.nz);
                    if (q < 0 || q >= nn) continue;
                }
                const int xq = cl.X(ax == 0 ? s : 0), yq = cl.Y(ax == 1 ? s : 0), zq = cl.Z(ax == 2 ? s : 0);
                const long long kb = bbox_index(a.g, b, xq, yq, zq);
                if (kb < 0) continue;
                const int kd = kind[kb];
                if (kd == 2) {
                    const long long nb = (long long)xq + (long long)a.g.nx * (yq + (long long)a.g.ny * zq);
                    for (int c = 0; c < 6; ++c) acc[c] += (double)tau[c * np + nb] / (double)nf_arr[kb];
                    touched = true;
                } else if (kd == 3) {
                    for (int c = 0; c < 6; ++c) acc[c] -= delta[c * nc + kb] / (double)nf_arr[kb];
                    touched = true;
                }
            }
            if (touched) {
                nf_arr[k] = 255;  // marks a stable cell whose stress changes
                for (int c = 0; c < 6; ++c) delta[c * nc + k] = acc[c];
            }
        }
        __syncthreads();
        // D: impulses and the populations of created cells.  A chunk of converted cells at a
        // time, one per thread, computes its momentum (deleted populations of a destroyed
        // cell; f^eq(rho_bar, u_b) of a created cell, whose populations it also writes) and
        // lever arm; thread 0 then adds them to the impulse in the sequential order of the
        // method: destroyed cells in cell order, then created cells in cell order.  A created
        // cell reads only stable cells' populations and writes only its own, so the cells of
        // a chunk are independent.
        double dP[3] = {0, 0, 0}, dL[3] = {0, 0, 0};
        for (int pass = 0; pass < 2; ++pass) {
            const int want = pass == 0 ? 2 : 3;
            for (int q0 = 0; q0 < nconv; q0 += blockDim.x) {
                const int q = q0 + (int)threadIdx.x;
                if (q < nconv && kind[conv[q]] == want) {
                    const long long k = conv[q];
                    int x, y, z;
                    const unsigned r = (unsigned)bbox_cell(a.g, b, k, x, y, z);
                    const Cell cl(a.g, x, y, z);
                    double Pm[3] = {0, 0, 0}, d[3];
                    min_image(a.g, P.X, x, y, z, d);
                    if (want == 2) {
                        R f[Q];
                        load_pdfs<S, PAR>(a, cl, r, f);
                        for (int c3 = 0; c3 < 3; ++c3)
                            for (int i = 0; i < Q; ++i) {
                                const double fi = (double)f[i] + (SH ? wgt<double>(i) * (double)a.ph.rho0 : 0.0);
                                Pm[c3] += fi * (double)cdir(i, c3);
                            }
                    } else {
                        double rsum = 0.0;
                        int cnt = 0;
                        for (int i = 1; i < Q; ++i) {
                            if (!a.g.per[0] && (x + cx(i) < 0 || x + cx(i) >= a.g.nx)) continue;
                            if (!a.g.per[1] && (y + cy(i) < 0 || y + cy(i) >= a.g.ny)) continue;
                            if (!a.g.per[2] && (z + cz(i) < 0 || z + cz(i) >= a.g.nz)) continue;
                            const int xq = cl.X(cx(i)), yq = cl.Y(cy(i)), zq = cl.Z(cz(i));
                            if (kind_of(b, xq, yq, zq) != 1) continue;
                            const unsigned nb =
                                (unsigned)xq + (unsigned)a.g.nx * ((unsigned)yq + (unsigned)a.g.ny * (unsigned)zq);
                            const Cell cn(a.g, xq, yq, zq);
                            R fn[Q];
                            load_pdfs<S, PAR>(a, cn, nb, fn);
                            double rn = 0.0;
                            for (int j = 0; j < Q; ++j) rn += (double)fn[j] + (SH ? wgt<double>(j) * (double)a.ph.rho0 : 0.0);
                            rsum += rn;
                            cnt++;
                        }
                        const double rho_bar = cnt > 0 ? rsum / (double)cnt : (double)a.ph.rho_ref;
                        double ub[3];
                        const double wxd[3] = {P.w[1] * d[2] - P.w[2] * d[1], P.w[2] * d[0] - P.w[0] * d[2],
                                               P.w[0] * d[1] - P.w[1] * d[0]};
                        for (int c3 = 0; c3 < 3; ++c3) ub[c3] = P.v[c3] + wxd[c3];
                        const double usq = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
                        double feq[Q];
                        for (int i = 0; i < Q; ++i) {
                            const double cu = cx(i) * ub[0] + cy(i) * ub[1] + cz(i) * ub[2];
                            feq[i] = wgt<double>(i) * rho_bar * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                        }
                        for (int i = 0; i < Q; ++i) {
                            S *dst = PAR == 0 ? a.f + (long long)i * np + r
                                              : a.f + (long long)copp(i) * np + cl.idx(-cx(i), -cy(i), -cz(i));
                            const double v = SH ? feq[i] - wgt<double>(i) * (double)a.ph.rho0 : feq[i];
                            Store<S>::st(dst, (R)v, a.ph.scale);
                        }
                        for (int c3 = 0; c3 < 3; ++c3)
                            for (int i = 0; i < Q; ++i) Pm[c3] += feq[i] * (double)cdir(i, c3);
                    }
                    for (int c3 = 0; c3 < 3; ++c3) {
                        s_pm[threadIdx.x][c3] = Pm[c3];
                        s_pm[threadIdx.x][3 + c3] = d[c3];
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int m = min((int)blockDim.x, nconv - q0);
                    for (int t = 0; t < m; ++t) {
                        const long long k = conv[q0 + t];
                        if (kind[k] != want) continue;
                        const double *Pm = s_pm[t], *d = s_pm[t] + 3;
                        if (want == 2) {
                            dP[0] += Pm[0];
                            dP[1] += Pm[1];
                            dP[2] += Pm[2];
                            dL[0] += d[1] * Pm[2] - d[2] * Pm[1];
                            dL[1] += d[2] * Pm[0] - d[0] * Pm[2];
                            dL[2] += d[0] * Pm[1] - d[1] * Pm[0];
                            if (nf_arr[k] == 0) {
                                int x, y, z;
                                const long long r = bbox_cell(a.g, b, k, x, y, z);
                                for (int c = 0; c < 6; ++c) diag[c] += (double)tau[c * np + r];
                            }
                            diag[6] += 1.0;
                        } else {
                            dP[0] -= Pm[0];
                            dP[1] -= Pm[1];
                            dP[2] -= Pm[2];
                            dL[0] -= d[1] * Pm[2] - d[2] * Pm[1];
                            dL[1] -= d[2] * Pm[0] - d[0] * Pm[2];
                            dL[2] -= d[0] * Pm[1] - d[1] * Pm[0];
                            diag[7] += 1.0;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x == 0)
            for (int c3 = 0; c3 < 3; ++c3) {
                P.dP[c3] = dP[c3];
                P.dL[c3] = dL[c3];
            }
        __syncthreads();
        // E: apply the stress moves and the new flags
        for (long long k = threadIdx.x; k < nc; k += blockDim.x) {
            const int kd = kind[k];
            if (kd == 0) continue;
            int x, y, z;
            const long long r = bbox_cell(a.g, b, k, x, y, z);
            if (kd == 1) {
                if (nf_arr[k] == 255)
                    for (int c = 0; c < 6; ++c) tau[c * np + r] = (R)((double)tau[c * np + r] + delta[c * nc + k]);
            } else if (kd == 3) {
                for (int c = 0; c < 6; ++c) tau[c * np + r] = (R)delta[c * nc + k];
                flag[r] = FLAG_FLUID;
            } else {
                for (int c = 0; c < 6; ++c) tau[c * np + r] = R(0);
                flag[r] = (uint8_t)(FLAG_PART0 + p);
            }
        }
        __syncthreads();
        // F: neighbour masks of the converted cells and their neighbours (the only cells
        // whose masks change; a cell reached twice gets the same value twice)
        for (int e = threadIdx.x; e < nconv * Q; e += blockDim.x) {
            const int q = e / Q, i = e - q * Q;
            int x, y, z;
            bbox_cell(a.g, b, conv[q], x, y, z);
            int xq = x + cx(i), yq = y + cy(i), zq = z + cz(i);
            if ((!a.g.per[0] && (xq < 0 || xq >= a.g.nx)) || (!a.g.per[1] && (yq < 0 || yq >= a.g.ny)) ||
                (!a.g.per[2] && (zq < 0 || zq >= a.g.nz)))
                continue;
            xq = wrapc(xq, a.g.nx);
            yq = wrapc(yq, a.g.ny);
            zq = wrapc(zq, a.g.nz);
            mask[(unsigned)xq + (unsigned)a.g.nx * ((unsigned)yq + (unsigned)a.g.ny * (unsigned)zq)] =
                cell_mask(a.g, flag, xq, yq, zq);
        }
        if (threadIdx.x == 0) {
            P.changed = 1;
            for (int c3 = 0; c3 < 3; ++c3) {
                P.v[c3] += P.dP[c3] / P.m;
                P.w[c3] += P.dL[c3] / P.I;
            }
        }
        // clear the stable-cell marks for the next particle / step
        for (long long k = threadIdx.x; k < nc; k += blockDim.x) nf_arr[k] = 0;
        __syncthreads();
    }
}
template <class S, int PAR>
__global__ void __launch_bounds__(512) k_fill_drain(KArgs<S> a, PartDev *__restrict__ parts, int nparts,
                                                    uint8_t *__restrict__ flag, uint32_t *__restrict__ mask,
                                                    typename Store<S>::R *__restrict__ tau,
                                                    uint8_t *__restrict__ kind, uint8_t *__restrict__ nf_arr,
                                                    double *__restrict__ delta, int *__restrict__ conv,
                                                    double *__restrict__ diag) {
    __shared__ double s_pm[512][6];  // per-thread momentum and lever arm of a converted cell
    fill_drain_block<S, PAR>(a, parts, nparts, flag, mask, tau, kind, nf_arr, delta, conv, diag, s_pm);
}

// Particle phase of a pool step for every member with particles, one 512-thread block per
// member: particle update, fill/drain, and the links of the particles whose cells
// converted -- the per-member code of the three separate kernels of a single solve, in
// the same order, so each member's results are those it gets alone.
template <class S>
struct PartEntry {
    KArgs<S> a[2];   // for even / odd steps k of a launch sequence (the stress ping-pong
                     // after the step's swap), pointers linked on the host
    int parity0;     // AA parity fill/drain works in at k = 0
    int nparts, first_seg;
    PartDev *parts;
    uint8_t *flag;
    uint32_t *mask;
    uint8_t *kind, *nf;
    double *delta, *diag;
    int *conv;
    long long *links;
    const int *seg_begin;
    int *seg_count;
    const int *capacity;
};
template <class S>
__global__ void __launch_bounds__(512) k_particle_phase_batched(const PartEntry<S> *__restrict__ e, int k) {
    using R = typename Store<S>::R;
    const PartEntry<S> &E = e[blockIdx.x];
    const KArgs<S> &a = E.a[k & 1];
    for (int p = (int)threadIdx.x; p < E.nparts; p += (int)blockDim.x) particle_update_one(E.parts[p]);
    __syncthreads();
    R *tau = const_cast<R *>(a.tau);
    __shared__ double s_pm[512][6];
    if (((E.parity0 + k) & 1) == 0)
        fill_drain_block<S, 0>(a, E.parts, E.nparts, E.flag, E.mask, tau, E.kind, E.nf, E.delta, E.conv, E.diag, s_pm);
    else
        fill_drain_block<S, 1>(a, E.parts, E.nparts, E.flag, E.mask, tau, E.kind, E.nf, E.delta, E.conv, E.diag, s_pm);
    __syncthreads();
    for (int p = 0; p < E.nparts; ++p) {
        particle_links_block<S, 512>(a.g, E.parts, p, E.flag, E.links, E.seg_begin, E.seg_count, E.first_seg,
                                     E.capacity);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// initialisation, read-back and reductions
// ---------------------------------------------------------------------------------

// f = f^eq(rho, u) of Eq. (lb-equilibrium) in the even-step layout; tau copied.  Works on
// the cells r0 .. r0+count-1; the inputs hold those cells with leading dimension ld.
template <class S>
__global__ void k_init(KArgs<S> a, const double *__restrict__ rho_in, const double *__restrict__ u_in,
                       const double *__restrict__ tau_in, typename Store<S>::R *__restrict__ tau_dst, long long r0,
                       long long count, long long ld) {
    using R = typename Store<S>::R;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const long long r = r0 + k;
    const double rho = rho_in ? rho_in[k] : (double)a.ph.rho_ref;
    double u[3] = {0.0, 0.0, 0.0};
    if (u_in)
        for (int j = 0; j < 3; ++j) u[j] = u_in[j * ld + k];
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double cu = (double)cx(i) * u[0] + (double)cy(i) * u[1] + (double)cz(i) * u[2];
        double v;
        if constexpr (!Store<S>::shifted) {
            v = wgt<double>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        } else {
            // deviation from w_i rho0, evaluated without forming f_i first
            v = wgt<double>(i) * ((rho - (double)a.ph.rho0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
        }
        Store<S>::st(a.f + (long long)i * a.g.np + r, (R)v, a.ph.scale);
    }
    double t6[6];
    const bool solid = a.mask[r] & 1u;  // a solid cell carries no stress
    for (int c = 0; c < 6; ++c) t6[c] = (tau_in && !solid) ? tau_in[c * ld + k] : 0.0;
    if (a.ph.fene && !solid) {
        // FENE-P: the conformation of the given stress, A = (I + lambda tau / eta_p) / f with
        // f = 1 + (3 + lambda tr tau / eta_p) / L^2
        const double lam = (double)a.ph.lam, eta_p = (double)a.ph.eta_p;
        const double s = 3.0 + lam * (t6[0] + t6[1] + t6[2]) / eta_p;
        const double f = 1.0 + s / (double)a.ph.fene_L2;
        for (int c = 0; c < 6; ++c) t6[c] = ((c < 3 ? 1.0 : 0.0) + lam * t6[c] / eta_p) / f;
    }
    for (int c = 0; c < 6; ++c) tau_dst[c * a.g.np + r] = (R)t6[c];
}

// rho, physical u and tau of the cells in z-planes z0.. (grid z extent), 0 in non-fluid
// cells; FP64 outputs indexed from the slab's first cell r0 with leading dimension ld.
template <class S, int PAR>
__global__ void k_read(KArgs<S> a, double *__restrict__ rho_out, double *__restrict__ u_out,
                       double *__restrict__ tau_out, int z0, long long ld) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.nx) return;
    const Cell cl(a.g, x, blockIdx.y, blockIdx.z + z0);
    const unsigned r = cl.self();
    const long long k = (long long)r - (long long)z0 * a.g.nx * a.g.ny;
    if (a.flag[r] != FLAG_FLUID) {
        if (rho_out) rho_out[k] = 0.0;
        for (int j = 0; j < 3; ++j)
            if (u_out) u_out[j * ld + k] = 0.0;
        for (int c = 0; c < 6; ++c)
            if (tau_out) tau_out[c * ld + k] = 0.0;
        return;
    }
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, a.ph, cl, r, a.mask[r], a.tau, Fp);
#pragma unroll
    for (int j = 0; j < 3; ++j) F[j] = a.ph.g[j] + Fp[j];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    if (rho_out) rho_out[k] = SH ? (double)a.ph.rho0 + (double)drho : (double)rho;
    for (int j = 0; j < 3; ++j)
        if (u_out) u_out[j * ld + k] = (double)u[j];
    if (tau_out) {
        R t6[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t6[c] = a.tau[c * a.g.np + r];
#pragma unroll
        for (int c = 0; c < 6; ++c) tau_out[c * ld + k] = (double)stored_to_stress<R>(a.ph, t6, c);
    }
}

// PDFs of every cell to / from unshifted FP64 in the plain (pre-collision) layout.
template <class S, int PAR>
__global__ void k_pdfs_io(KArgs<S> a, double *__restrict__ io, int write) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.nx) return;
    const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
    const unsigned r = cl.self();
    const long long np = a.g.np, n = a.g.n;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        S *p = PAR == 0 ? a.f + (long long)i * np + r : a.f + (long long)copp(i) * np + cl.idx(-cx(i), -cy(i), -cz(i));
        const double base = Store<S>::shifted ? wgt<double>(i) * (double)a.ph.rho0 : 0.0;
        if (write) {
            Store<S>::st(p, (typename Store<S>::R)(io[i * n + r] - base), a.ph.scale);
        } else {
            io[i * n + r] = base + (double)Store<S>::ld(p, a.ph.inv_scale);
        }
    }
}

// Probe listed cells: 19 unshifted PDFs, rho, physical u, tau (29 doubles per cell).
template <class S, int PAR>
__global__ void k_probe(KArgs<S> a, const long long *__restrict__ cells, int count, double *__restrict__ out) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const unsigned r = (unsigned)cells[k];
    const int x = (int)(r % a.g.nx), y = (int)((r / a.g.nx) % a.g.ny), z = (int)(r / ((unsigned)a.g.nx * a.g.ny));
    const Cell cl(a.g, x, y, z);
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    double *o = out + (long long)k * 29;
    for (int i = 0; i < Q; ++i) o[i] = (double)f[i] + (SH ? wgt<double>(i) * (double)a.ph.rho0 : 0.0);
    for (int j = 19; j < 29; ++j) o[j] = 0.0;
    if (a.flag[r] != FLAG_FLUID) return;
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, a.ph, cl, r, a.mask[r], a.tau, Fp);
    for (int j = 0; j < 3; ++j) F[j] = a.ph.g[j] + Fp[j];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    o[19] = SH ? (double)a.ph.rho0 + (double)drho : (double)rho;
    for (int j = 0; j < 3; ++j) o[20 + j] = (double)u[j];
    R t6[6];
    for (int c = 0; c < 6; ++c) t6[c] = a.tau[c * a.g.np + r];
    for (int c = 0; c < 6; ++c) o[23 + c] = (double)stored_to_stress<R>(a.ph, t6, c);
}

// Per-block FP64 partial sums over fluid cells: mass, momentum, count, bad-value flag.
template <class S, int PAR>
__global__ void __launch_bounds__(256) k_reduce(KArgs<S> a, double *__restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (x < a.g.nx) {
        const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
        const unsigned r = cl.self();
        if (a.flag[r] == FLAG_FLUID && (int)blockIdx.z >= a.zlo && (int)blockIdx.z < a.zhi) {
            typename Store<S>::R f[Q];
            load_pdfs<S, PAR>(a, cl, r, f);
            for (int i = 0; i < Q; ++i) {
                const double fi = (double)f[i] + (Store<S>::shifted ? wgt<double>(i) * (double)a.ph.rho0 : 0.0);
                v[0] += fi;
                v[1] += cx(i) * fi;
                v[2] += cy(i) * fi;
                v[3] += cz(i) * fi;
                if (!isfinite(fi)) v[5] = 1.0;
            }
            v[4] = 1.0;
            if (!(v[0] > 0.0)) v[5] = 1.0;
        }
    }
    __shared__ double sh[6][256];
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 6; ++k)
                sh[k][threadIdx.x] = k == 5 ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + s])
                                            : sh[k][threadIdx.x] + sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        for (int k = 0; k < 6; ++k) partial[b * 6 + k] = sh[k][0];
    }
}

// ---------------------------------------------------------------------------------
// z-slab decomposition: halo exchange between the slabs of one domain.  A slab computes
// planes [zlo, zhi) and holds one ghost plane on each side (zlo - 1, zhi) mirroring the
// neighbouring slab's boundary plane (its flags included).  Per step:
//   after the stream-collide: u of the boundary planes -> the neighbours' ghost planes,
//     and the 5 PDFs per cell that cross each face (below);
//   after the stress update: tau of the boundary planes -> the neighbours' ghost planes.
// The PDFs follow the in-place (AA) pattern.  D+ / D- are the directions with c_z = +1 /
// -1 (5 each).  After an even step a fluid cell's slot -i holds its f*_i, which the next
// odd step reads from the cell above (-i in D-, i moving up) or below: the boundary
// plane's slots D- (high side) / D+ (low side) go into the neighbour's ghost plane, for
// fluid ghost cells (a solid ghost cell's slots hold this slab's own bounced values).
// After an odd step a fluid cell has written f*_i into slot i of r + c_i, in the ghost
// plane for i crossing the face: the ghost plane's slots D+ (high side) / D- (low side)
// go into the neighbour's boundary plane, where the source cell r - c_i is fluid (else
// the slot holds that cell's own bounced value).
// ---------------------------------------------------------------------------------
__host__ __device__ constexpr int dir_zp(int k) { return k == 0 ? 5 : k == 1 ? 11 : k == 2 ? 14 : k == 3 ? 15 : 18; }
__host__ __device__ constexpr int dir_zm(int k) { return k == 0 ? 6 : k == 1 ? 12 : k == 2 ? 13 : k == 3 ? 16 : 17; }

__host__ __device__ constexpr int halo_values(int what) { return what == 0 ? 5 : (what == 1 ? 3 : 6); }

// plane and slot set of a PDF pack (side: 0 low, 1 high; parity of the last stream-collide)
__device__ __forceinline__ void halo_f_pack_plan(int side, int parity, int zlo, int zhi, int &z, bool &up) {
    if (parity == 0) {
        z = side ? zhi - 1 : zlo;
        up = side == 0;  // low side sends D+, high side D-
    } else {
        z = side ? zhi : zlo - 1;
        up = side == 1;  // from the ghost planes: high sends D+, low D-
    }
}

template <class S>
__global__ void k_halo_pack(KArgs<S> a, int what, int side, int parity, void *__restrict__ buf) {
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.g.nx) return;
    const long long plane = (long long)a.g.nx * a.g.ny, p = x + (long long)a.g.nx * y;
    const size_t np = (size_t)a.g.np;
    if (what == 0) {
        int z;
        bool up;
        halo_f_pack_plan(side, parity, a.zlo, a.zhi, z, up);
        const unsigned r = (unsigned)(p + plane * z);
        S *o = (S *)buf;
#pragma unroll
        for (int k = 0; k < 5; ++k) o[k * plane + p] = a.f[(up ? dir_zp(k) : dir_zm(k)) * np + r];
    } else {
        const int z = side ? a.zhi - 1 : a.zlo;
        const unsigned r = (unsigned)(p + plane * z);
        R *o = (R *)buf;
        if (what == 1)
            for (int j = 0; j < 3; ++j) o[j * plane + p] = a.u_out[j * np + r];
        else
            for (int c = 0; c < 6; ++c) o[c * plane + p] = a.tau[c * np + r];
    }
}

template <class S>
__global__ void k_halo_unpack(KArgs<S> a, int what, int side, int parity, const void *__restrict__ buf) {
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.g.nx) return;
    const long long plane = (long long)a.g.nx * a.g.ny, p = x + (long long)a.g.nx * y;
    const size_t np = (size_t)a.g.np;
    if (what == 0) {
        const S *in = (const S *)buf;
        if (parity == 0) {
            // into the ghost plane, for fluid ghost cells; the low side receives the lower
            // slab's D-, the high side the upper slab's D+
            const int z = side ? a.zhi : a.zlo - 1;
            const unsigned r = (unsigned)(p + plane * z);
            if (a.flag[r] != FLAG_FLUID) return;
#pragma unroll
            for (int k = 0; k < 5; ++k) a.f[(side ? dir_zp(k) : dir_zm(k)) * np + r] = in[k * plane + p];
        } else {
            // into the boundary plane, where the source cell r - c_i (in the ghost plane) is
            // fluid: the low side receives D+ (moving up from the lower slab), the high
            // side D- (moving down from the upper slab)
            const int z = side ? a.zhi - 1 : a.zlo;
            const unsigned r = (unsigned)(p + plane * z);
            const Cell cl(a.g, x, y, z);
            if (a.flag[r] != FLAG_FLUID) return;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int i = side ? dir_zm(k) : dir_zp(k);
                const int sx = -cx(i), sy = -cy(i);
                const int xs = x + sx, ys = y + sy;
                if ((xs < 0 || xs >= a.g.nx) && !a.g.per[0]) continue;
                if ((ys < 0 || ys >= a.g.ny) && !a.g.per[1]) continue;
                if (a.flag[cl.idx(sx, sy, -cz(i))] != FLAG_FLUID) continue;
                a.f[i * np + r] = in[k * plane + p];
            }
        }
    } else {
        const int z = side ? a.zhi : a.zlo - 1;
        const unsigned r = (unsigned)(p + plane * z);
        const R *in = (const R *)buf;
        if (what == 1)
            for (int j = 0; j < 3; ++j) a.u_out[j * np + r] = in[j * plane + p];
        else
            for (int c = 0; c < 6; ++c) const_cast<R *>(a.tau)[c * np + r] = in[c * plane + p];
    }
}

} // namespace lbve

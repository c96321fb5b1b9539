// lbve_device.cuh -- device-side building blocks of the coupled LB + Oldroyd-B step
// (Kuron et al., arXiv:2009.12279): D3Q19 lattice, PDF storage codecs, boundary
// velocities, the TRT collision with Guo forcing, the polymer force and the
// finite-volume stress update.  Included by the per-precision kernel translation units.
//
// Storage: PDFs are structure-of-arrays, 19 arrays of `np` cells (np = n padded to a
// multiple of 64), updated in place with the AA pattern: on an even step every cell
// reads its own slots and writes the post-collision f*_i into its own slot -i; on an
// odd step it reads f_i from slot -i of cell r - c_i and writes f*_i into slot i of
// r + c_i.  Both steps touch every PDF once for reading and once for writing, half the
// traffic of a two-array scheme.  A population that would stream into a solid cell is
// bounced back (Eq. (ubb)) into the slot the next step reads it from; solid cells'
// slots serve as the ghost storage for those bounced populations.
//
// Precision: FP64 storage keeps f_i itself and every formula is evaluated in the same
// operation order as the plain statement of the paper's equations (the FP64 build has
// FMA contraction off), so the FP64 mode reproduces a plain IEEE evaluation.  The FP32,
// FP16 and BF16 storage modes keep the deviation (f_i - w_i rho0) * 2^k and do all
// arithmetic in FP32 on deviations (rho = rho0 + sum of deviations).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbve_launch.h"

namespace lbve {

// --------------------------------------------------------------------------------
// D3Q19 velocity set (Sec. "Lattice Boltzmann"), packed two bits per direction so
// that the component lookups fold to constants inside unrolled loops.
// --------------------------------------------------------------------------------
constexpr int kCX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kCY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kCZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

constexpr uint64_t pack_dirs(const int (&c)[Q]) {
    uint64_t m = 0;
    for (int i = 0; i < Q; ++i) m |= (uint64_t)(c[i] + 1) << (2 * i);
    return m;
}
constexpr uint64_t kPX = pack_dirs(kCX), kPY = pack_dirs(kCY), kPZ = pack_dirs(kCZ);

__host__ __device__ __forceinline__ constexpr int cx(int i) { return (int)((kPX >> (2 * i)) & 3u) - 1; }
__host__ __device__ __forceinline__ constexpr int cy(int i) { return (int)((kPY >> (2 * i)) & 3u) - 1; }
__host__ __device__ __forceinline__ constexpr int cz(int i) { return (int)((kPZ >> (2 * i)) & 3u) - 1; }
__host__ __device__ __forceinline__ constexpr int copp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ __forceinline__ constexpr int cdir(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }

template <class R>
__host__ __device__ __forceinline__ constexpr R wgt(int i) {
    return i == 0 ? R(1.0 / 3.0) : (i < 7 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}

// symmetric tensor component of (a, b) in the layout xx, yy, zz, xy, xz, yz
__host__ __device__ __forceinline__ constexpr int comp(int a, int b) {
    return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}
__host__ __device__ __forceinline__ constexpr int comp_i(int c) { return c < 3 ? c : (c == 5 ? 1 : 0); }
__host__ __device__ __forceinline__ constexpr int comp_j(int c) { return c < 3 ? c : (c == 3 ? 1 : 2); }

// --------------------------------------------------------------------------------
// PDF storage codecs
// --------------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
    using R = double;
    static constexpr bool shifted = false;
    static constexpr bool keyed = false;
    __device__ static __forceinline__ double ld(const double *p, double) { return *p; }
    __device__ static __forceinline__ void st(double *p, double v, double) { *p = v; }
};
template <>
struct Store<float> {
    using R = float;
    static constexpr bool shifted = true;
    static constexpr bool keyed = false;
    // FP32 keeps its exponent range: stored unscaled (the scale argument is 1)
    __device__ static __forceinline__ float ld(const float *p, float) { return *p; }
    __device__ static __forceinline__ void st(float *p, float v, float) { *p = v; }
};
// The 16-bit modes round the stream-collide's stores stochastically: with 8 (BF16) or 11
// (FP16) significant bits, the per-step change of a slowly evolving flow can be below half
// a unit of the stored deviation, and round-to-nearest would drop it every step (the flow
// stalls).  Stochastic rounding rounds up with probability equal to the dropped fraction
// (unbiased).  Blackwell converts two FP32 values at once with it (cvt.rs, one instruction
// per pair): the first value goes to the high half of the result, rounded with the high
// 16 of the 32 random bits, the second to the low half with the low 16.  The random bits
// come from a counter-based hash of (step, cell, direction), so results are deterministic
// and the same for a solve alone and in a pool.  round2 returns the pair; store16 writes
// one half.
template <>
struct Store<__half> {
    using R = float;
    static constexpr bool shifted = true;
    static constexpr bool keyed = true;
    __device__ static __forceinline__ float ld(const __half *p, float inv) { return __half2float(*p) * inv; }
    __device__ static __forceinline__ void st(__half *p, float v, float sc) { *p = __float2half_rn(v * sc); }
    __device__ static __forceinline__ uint32_t round2(float a, float b, float sc, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a * sc), "f"(b * sc), "r"(rbits));
        return d;
    }
    __device__ static __forceinline__ void store16(__half *p, uint32_t bits) {
        *reinterpret_cast<unsigned short *>(p) = (unsigned short)bits;
    }
};
template <>
struct Store<__nv_bfloat16> {
    using R = float;
    static constexpr bool shifted = true;
    static constexpr bool keyed = true;
    // BF16 has the FP32 exponent range: stored unscaled (the scale argument is 1)
    __device__ static __forceinline__ float ld(const __nv_bfloat16 *p, float) { return __bfloat162float(*p); }
    __device__ static __forceinline__ void st(__nv_bfloat16 *p, float v, float) { *p = __float2bfloat16_rn(v); }
    __device__ static __forceinline__ uint32_t round2(float a, float b, float, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
        return d;
    }
    __device__ static __forceinline__ void store16(__nv_bfloat16 *p, uint32_t bits) {
        *reinterpret_cast<unsigned short *>(p) = (unsigned short)bits;
    }
};

// Counter-based random bits: the 32-bit finaliser of MurmurHash3 (A. Appleby) over a cell
// and step key, uniform in all 32 bits; each pair of directions takes it xor a distinct
// constant (one instruction).  Every rounding stays unbiased (each half of the bits is
// uniform); only the pairs' bits are related within a cell.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ uint32_t pair_bits(uint32_t h, int p) { return h ^ ((uint32_t)(p + 1) * 0x9E3779B9u); }

// Coordinates of one cell and its periodically wrapped neighbours; cell indices are
// 32-bit (grids are limited to 2^31 cells).
struct Cell {
    int x, y, z;
    int xm, xp, ym, yp, zm, zp;
    unsigned nx, nxy;
    __device__ __forceinline__ Cell(const Geo &g, int x_, int y_, int z_) : x(x_), y(y_), z(z_) {
        xm = x == 0 ? g.nx - 1 : x - 1;
        xp = x == g.nx - 1 ? 0 : x + 1;
        ym = y == 0 ? g.ny - 1 : y - 1;
        yp = y == g.ny - 1 ? 0 : y + 1;
        zm = z == 0 ? g.nz - 1 : z - 1;
        zp = z == g.nz - 1 ? 0 : z + 1;
        nx = (unsigned)g.nx;
        nxy = (unsigned)g.nx * (unsigned)g.ny;
    }
    __device__ __forceinline__ int X(int d) const { return d == 0 ? x : (d > 0 ? xp : xm); }
    __device__ __forceinline__ int Y(int d) const { return d == 0 ? y : (d > 0 ? yp : ym); }
    __device__ __forceinline__ int Z(int d) const { return d == 0 ? z : (d > 0 ? zp : zm); }
    __device__ __forceinline__ unsigned idx(int dx, int dy, int dz) const {
        return (unsigned)X(dx) + nx * (unsigned)Y(dy) + nxy * (unsigned)Z(dz);
    }
    __device__ __forceinline__ unsigned self() const { return (unsigned)x + nx * (unsigned)y + nxy * (unsigned)z; }
};

// Neighbour mask of a cell: bit 0 set if the cell is not fluid, bit i (1..18) set if the
// neighbour r + c_i is not fluid, MASK_MOVING set if one of those neighbours is a wall
// class or a particle cell (a boundary that may move, Eq. (ubb)) rather than a resting
// no-slip wall.  Faces of the D3Q7 set are directions 1..6.
constexpr uint32_t MASK_MOVING = 1u << 19;
__device__ __forceinline__ bool nb_solid(uint32_t m, int i) { return (m >> i) & 1u; }

// --------------------------------------------------------------------------------
// Lane arithmetic of the shifted modes (FP32 arithmetic on deviations).  Every operation
// rounds once and none is left to the compiler to contract, so a cell computed in a float
// and two cells computed in the two lanes of a float2 (Blackwell's paired FP32
// instructions: two FMAs, adds or multiplies per instruction) give bitwise the same
// results.  Masks are a uint32_t for one cell and a uint2 for two.
// --------------------------------------------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class V>
__device__ __forceinline__ V vbc(float s);
template <>
__device__ __forceinline__ float vbc<float>(float s) { return s; }
template <>
__device__ __forceinline__ float2 vbc<float2>(float s) { return make_float2(s, s); }
// correctly rounded reciprocal (no paired form: one per lane)
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
__device__ __forceinline__ float vdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float2 vdiv(float2 a, float2 b) { return make_float2(__fdiv_rn(a.x, b.x), __fdiv_rn(a.y, b.y)); }
// select per lane: if_solid where neighbour i of the lane's cell is not fluid
__device__ __forceinline__ float vsel_solid(uint32_t m, int i, float if_solid, float if_fluid) {
    return nb_solid(m, i) ? if_solid : if_fluid;
}
__device__ __forceinline__ float2 vsel_solid(uint2 m, int i, float2 if_solid, float2 if_fluid) {
    return make_float2(nb_solid(m.x, i) ? if_solid.x : if_fluid.x, nb_solid(m.y, i) ? if_solid.y : if_fluid.y);
}

// Boundary velocity u_b of the solid cell (xq, yq, zq) with flag fl: zero for a no-slip
// wall, the class velocity for a moving wall (Eq. (ubb)), v + w x (r_b - X) with the
// minimum-image lever arm for a particle cell (Eq. (surface-velocity)).
template <class R>
__device__ __forceinline__ void boundary_velocity(const Geo &g, const Phys<R> &ph, const PartDev *parts, int fl,
                                                  int xq, int yq, int zq, R ub[3]) {
    ub[0] = R(0);
    ub[1] = R(0);
    ub[2] = R(0);
    if (fl >= FLAG_WALL0 && fl < FLAG_WALL0 + MAX_WALL) {
        ub[0] = ph.wall_vel[fl - FLAG_WALL0][0];
        ub[1] = ph.wall_vel[fl - FLAG_WALL0][1];
        ub[2] = ph.wall_vel[fl - FLAG_WALL0][2];
    } else if (fl >= FLAG_PART0 && fl < FLAG_PART0 + MAX_PART) {
        const PartDev &P = parts[fl - FLAG_PART0];
        double q[3] = {(double)xq, (double)yq, (double)zq};
        int nn[3] = {g.nx, g.ny, g.nz};
        double d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[a] = q[a] - P.X[a];
            if (g.per[a]) d[a] -= (double)nn[a] * floor(d[a] / (double)nn[a] + 0.5);
        }
        ub[0] = (R)(P.v[0] + (P.w[1] * d[2] - P.w[2] * d[1]));
        ub[1] = (R)(P.v[1] + (P.w[2] * d[0] - P.w[0] * d[2]));
        ub[2] = (R)(P.v[2] + (P.w[0] * d[1] - P.w[1] * d[0]));
    }
}

// Boundary velocity with the common no-slip case inline and the moving-wall / particle
// cases out of line (they are rare and would otherwise bloat every caller).
template <class R>
struct Vec3 {
    R x, y, z;
};
// Out-of-line wall-class / particle branch of boundary_velocity; the result comes back by
// value so that callers keep their velocity arrays in registers.
template <class R>
__device__ __noinline__ Vec3<R> boundary_velocity_slow(const Geo &g, const Phys<R> &ph, const PartDev *parts, int fl,
                                                       int xq, int yq, int zq) {
    R t[3];
    boundary_velocity<R>(g, ph, parts, fl, xq, yq, zq, t);
    return Vec3<R>{t[0], t[1], t[2]};
}

// boundary_velocity with the resting no-slip case inline.
template <class R>
__device__ __forceinline__ void boundary_velocity_fast(const Geo &g, const Phys<R> &ph, const PartDev *parts, int fl,
                                                       int xq, int yq, int zq, R ub[3]) {
    if (fl == FLAG_NOSLIP) {
        ub[0] = R(0);
        ub[1] = R(0);
        ub[2] = R(0);
    } else {
        const Vec3<R> v = boundary_velocity_slow<R>(g, ph, parts, fl, xq, yq, zq);
        ub[0] = v.x;
        ub[1] = v.y;
        ub[2] = v.z;
    }
}

// --------------------------------------------------------------------------------
// local operators
// --------------------------------------------------------------------------------

// Polymer force Eq. (force) on the D3Q7 faces (A_0 = 1): F_j = sum_faces s tau_kj(face),
// face value by Eq. (interpolation), or tau(r) towards a solid cell (Eq. (extrapolation)).
// tn(l, c) returns component c of the stress of the face-l neighbour (l = 0..5 for
// +x, -x, +y, -y, +z, -z); it is only called for fluid neighbours.
// Shifted modes: the two faces of an axis share the cell's own stress, which cancels:
// F_j = sum_k 1/2 (a_kj - b_kj), a = tau_kj(r + e_k) (tau_kj(r) when r + e_k is solid), b
// likewise on the -e_k side.  V = float (one cell) or float2 (two cells), M its mask type.
template <class V, class M, class TauNb>
__device__ __forceinline__ void polymer_force_sh(const V (&tr)[6], M mask, const TauNb &tn, V Fp[3]) {
    const V half = vbc<V>(0.5f);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        V acc;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = comp(k, j);
            const V a = vsel_solid(mask, 2 * k + 1, tr[c], tn(2 * k, c));
            const V b = vsel_solid(mask, 2 * k + 2, tr[c], tn(2 * k + 1, c));
            const V d = vsub(a, b);
            acc = k == 0 ? vmul(half, d) : vfma(half, d, acc);
        }
        Fp[j] = acc;
    }
}

template <class R, class TauNb>
__device__ __forceinline__ void polymer_force_core(const R (&tr)[6], uint32_t mask, const TauNb &tn, R Fp[3]) {
    if constexpr (sizeof(R) == 4) {
        polymer_force_sh<float>(tr, mask, tn, Fp);
        return;
    }
    Fp[0] = R(0);
    Fp[1] = R(0);
    Fp[2] = R(0);
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        const int k = l >> 1;
        const int s = (l & 1) ? -1 : 1;
        const bool fl = !nb_solid(mask, l + 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int c = comp(k, j);
            const R tf = fl ? R(0.5) * (tr[c] + tn(l, c)) : tr[c];
            if (s > 0)
                Fp[j] = Fp[j] + tf;
            else
                Fp[j] = Fp[j] - tf;
        }
    }
}

// FENE-P closure (the conformation tensor A in the stress arrays): the stress component c
// of a cell, tau_c = (eta_p / lambda)(f A_c - delta_c), f = 1 / (1 - tr A / L^2).
template <class R>
__device__ __forceinline__ R fene_factor(const Phys<R> &ph, R a0, R a1, R a2) {
    return R(1) / (R(1) - ((a0 + a1) + a2) / ph.fene_L2);
}
template <class R>
__device__ __forceinline__ R fene_component(const Phys<R> &ph, R f, R a, int c) {
    return c < 3 ? ph.ep_l * (f * a - R(1)) : ph.ep_l * (f * a);
}

// Eq. (force) as polymer_force_core, with the stress of each cell computed from its
// conformation tensor (FENE-P).  tn(l, c) returns component c of the face-l neighbour's A;
// besides the face's row it reads the neighbour's diagonal for the trace.
template <class R, class TauNb>
__device__ __forceinline__ void polymer_force_core_fene(const R (&tr)[6], uint32_t mask, const TauNb &tn,
                                                        const Phys<R> &ph, R Fp[3]) {
    const R fr = fene_factor<R>(ph, tr[0], tr[1], tr[2]);
    R ts[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) ts[c] = fene_component<R>(ph, fr, tr[c], c);
    Fp[0] = R(0);
    Fp[1] = R(0);
    Fp[2] = R(0);
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        const int k = l >> 1;
        const int s = (l & 1) ? -1 : 1;
        const bool fl = !nb_solid(mask, l + 1);
        R fn = R(0);
        if (fl) fn = fene_factor<R>(ph, tn(l, 0), tn(l, 1), tn(l, 2));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int c = comp(k, j);
            const R tf = fl ? R(0.5) * (ts[c] + fene_component<R>(ph, fn, tn(l, c), c)) : ts[c];
            if (s > 0)
                Fp[j] = Fp[j] + tf;
            else
                Fp[j] = Fp[j] - tf;
        }
    }
}

// Same with the stress read from global memory (the FENE-P form when ph.fene).
template <class R>
__device__ __forceinline__ void polymer_force(const Geo &g, const Phys<R> &ph, const Cell &cl, unsigned r,
                                              uint32_t mask, const R *__restrict__ tau, R Fp[3]) {
    const size_t np = (size_t)g.np;
    R tr[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) tr[c] = tau[c * np + r];
    auto tn = [&](int l, int c) -> R {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        return tau[c * np + cl.idx(k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0)];
    };
    if (ph.fene)
        polymer_force_core_fene<R>(tr, mask, tn, ph, Fp);
    else
        polymer_force_core<R>(tr, mask, tn, Fp);
}

// Stress of a cell's stored tensor (itself, or the FENE-P stress of a conformation).
template <class R>
__device__ __forceinline__ R stored_to_stress(const Phys<R> &ph, const R (&a)[6], int c) {
    if (!ph.fene) return a[c];
    return fene_component<R>(ph, fene_factor<R>(ph, a[0], a[1], a[2]), a[c], c);
}

// Macroscopic moments of the shifted modes (deviations: rho = rho0 + sum), lane form.
template <class V>
__device__ __forceinline__ void moments_sh(const V (&f)[Q], const V F[3], float rho0, V &rho, V &drho, V u[3]) {
    const V d0 = vadd(vadd(vadd(vadd(f[0], f[1]), vadd(f[2], f[3])), vadd(f[4], f[5])), f[6]);
    const V d1 = vadd(vadd(vadd(f[7], f[8]), vadd(f[9], f[10])), vadd(f[11], f[12]));
    const V d2 = vadd(vadd(vadd(f[13], f[14]), vadd(f[15], f[16])), vadd(f[17], f[18]));
    drho = vadd(vadd(d0, d1), d2);
    rho = vadd(vbc<V>(rho0), drho);
    const V m78 = vsub(f[7], f[8]), m1112 = vsub(f[11], f[12]), m1516 = vsub(f[15], f[16]);
    const V m910 = vsub(f[9], f[10]), m1314 = vsub(f[13], f[14]), m1718 = vsub(f[17], f[18]);
    // jx = c_x-weighted sum, jy, jz likewise (pairs (i, -i) differenced first)
    const V jx = vadd(vadd(vadd(vadd(vsub(f[1], f[2]), m78), m910), m1112), m1314);
    const V jy = vadd(vadd(vsub(vadd(vsub(f[3], f[4]), m78), m910), m1516), m1718);
    const V jz = vsub(vadd(vsub(vadd(vsub(f[5], f[6]), m1112), m1314), m1516), m1718);
    const V ir = vrcp(rho);
    const V half = vbc<V>(0.5f);
    u[0] = vmul(vfma(half, F[0], jx), ir);
    u[1] = vmul(vfma(half, F[1], jy), ir);
    u[2] = vmul(vfma(half, F[2], jz), ir);
}

// Macroscopic moments, Eq. (macroscopic-velocity).  FP64 mode sums in direction order;
// shifted modes return rho = rho0 + drho with drho summed over the deviations.
template <class R, bool SH>
__device__ __forceinline__ void moments(const R (&f)[Q], const R F[3], R rho0, R &rho, R &drho, R u[3]) {
    if constexpr (!SH) {
        R s = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) s = s + f[i];
        R j[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R t = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int c = cdir(i, a);
                if (c == 1) t = t + f[i];
                if (c == -1) t = t - f[i];
            }
            j[a] = t;
        }
        rho = s;
        drho = s;
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + R(0.5) * F[a]) / s;
    } else {
        moments_sh<R>(f, F, rho0, rho, drho, u);
    }
}

// c_i . v for a direction with components in {-1,0,1}, in the order x, y, z.
template <class R>
__device__ __forceinline__ R cdot(int i, const R v[3]) {
    R t = R(0);
    bool first = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c = cdir(i, a);
        if (c != 0) {
            if (first) {
                t = c > 0 ? v[a] : -v[a];
                first = false;
            } else {
                t = c > 0 ? t + v[a] : t - v[a];
            }
        }
    }
    return t;
}

// TRT collision with Guo forcing, Eqs. (lb), (lb-equilibrium), (guo), in place on f.
// FP64 mode: feq_i = (w_i rho)(1 + 3 cu + 9/2 cu^2 - 3/2 u^2), each population evaluated
// as the plain statement of the equations orders it.  Shifted modes work on the
// deviations, with feq_i - w_i rho0 = w_i (drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)), and
// fold the pair (i, -i) algebraically:
//   f*_{+-i} = f_{+-i} - P -+ M,
//   P = omega+/(2 k2) (k2 (f_i + f_-i) - (drho + rho (9/2 cu^2 - 3/2 u^2))) - w_i B (9 cu cF - 3 u.F)
//   M = omega-/(2 k)  (k  (f_i - f_-i) - rho cu)                           - w_i A cF
// with k = 1/(6 w_i) and k2 = 1/(2 w_i), small integers (3 and 9 for w = 1/18, 6 and 18 for
// w = 1/36).  The non-equilibrium parts are formed first, by an exact integer multiple inside
// one fused multiply-add, and only then scaled by a rounded constant.  Scaling the large
// antisymmetric equilibrium 3 w_i rho cu by rounded FP32 weights instead makes the lattice
// sum of the relaxed momentum differ from rho u by a fixed relative ~3e-8 every step: a
// systematic momentum drift that, in a flow accelerating from rest, grows linearly in time
// (relative error 1.1e-5 after 1000 steps of the config-1 channel, against 1.3e-7 in this form).
// Returns true when the cell is unstable: rho <= 0, |u|^2 >= 1/3 (the lattice sound speed
// squared) or a NaN in either (comparisons with a NaN are false).
// c_i . v of the directions i = 1, 3, ..., 17 (the first of each pair (i, -i)), lane form:
// one component or the sum / difference of two
template <class V>
__device__ __forceinline__ V cdot_v(int i, const V v[3]) {
    int a = -1, b = -1, sb = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = cdir(i, k);
        if (c != 0) {
            if (a < 0) {
                a = k;
            } else {
                b = k;
                sb = c;
            }
        }
    }
    if (b < 0) return v[a];  // the first direction of a pair has its one component +1
    return sb > 0 ? vadd(v[a], v[b]) : vsub(v[a], v[b]);
}

// Collision of the shifted modes in lane form (see collide): the non-equilibrium parts of
// each pair are formed first, k2 (f_i + f_-i) - esym and k (f_i - f_-i) - rho c.u, each
// in one fused multiply-add with the exact integer k2 = 1/(2 w_i) or k = 1/(6 w_i), and
// only then scaled by rounded rates.  Returns the instability test per lane.
template <class V>
struct LaneBool;
template <>
struct LaneBool<float> {
    using T = bool;
};
template <>
struct LaneBool<float2> {
    using T = uint2;  // x, y: 1 when that lane's cell is unstable
};
__device__ __forceinline__ bool unstable_of(float rho, float usq) {
    return !(rho > 0.0f) || !(usq < (float)(1.0 / 3.0));
}
__device__ __forceinline__ uint2 unstable_of(float2 rho, float2 usq) {
    return make_uint2(unstable_of(rho.x, usq.x) ? 1u : 0u, unstable_of(rho.y, usq.y) ? 1u : 0u);
}
template <class V>
__device__ __forceinline__ typename LaneBool<V>::T collide_sh(V (&f)[Q], V rho, V drho, const V u[3], const V F[3],
                                                             const Phys<float> &ph) {
    const V usq = vfma(u[2], u[2], vfma(u[0], u[0], vmul(u[1], u[1])));
    const auto unstable = unstable_of(rho, usq);
    const V uF = vfma(u[2], F[2], vfma(u[0], F[0], vmul(u[1], F[1])));
    const float wp = ph.omega_p, wm = ph.omega_m;
    const V q = vmul(vbc<V>(1.5f), usq);
    const V u3F = vmul(vbc<V>(3.0f), uF);
    // omega+/(2 k2) and omega-/(2 k) of the directions with w = 1/18 (halved for 1/36);
    // these rounded constants scale only the small non-equilibrium parts
    const float cp = wp * (float)(1.0 / 18.0), cm = wm * (float)(1.0 / 6.0);
    // rest population: feq0 - w0 rho0 = w0 (drho - rho q), forcing w0 B (-3 u.F)
    {
        const float w0 = wgt<float>(0);
        const V e0 = vfma(vneg(rho), q, drho);
        const V n0 = vfma(vbc<V>(-w0), e0, f[0]);
        f[0] = vfma(vbc<V>(-(w0 * ph.B)), u3F, vfma(vbc<V>(-wp), n0, f[0]));
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int ip = i + 1;
        const bool axis = i < 7;  // w = 1/18
        const float w = wgt<float>(i);
        const float k = axis ? 3.0f : 6.0f, k2 = axis ? 9.0f : 18.0f;
        const float sp = axis ? cp : 0.5f * cp, sm = axis ? cm : 0.5f * cm;
        const V cu = cdot_v<V>(i, u);
        const V cF = cdot_v<V>(i, F);
        const V esym = vfma(rho, vfma(vmul(vbc<V>(4.5f), cu), cu, vneg(q)), drho);
        const V x9 = vfma(vmul(vbc<V>(9.0f), cu), cF, vneg(u3F));
        const V nsym = vfma(vbc<V>(k2), vadd(f[i], f[ip]), vneg(esym));       // k2 (f_i + f_-i) - esym
        const V nanti = vfma(vbc<V>(k), vsub(f[i], f[ip]), vneg(vmul(rho, cu)));  // k (f_i - f_-i) - rho cu
        const V P = vfma(vbc<V>(-(w * ph.B)), x9, vmul(vbc<V>(sp), nsym));
        const V M = vfma(vbc<V>(-(w * ph.A)), cF, vmul(vbc<V>(sm), nanti));
        const V fi = vsub(vsub(f[i], P), M);
        const V fo = vadd(vsub(f[ip], P), M);
        f[i] = fi;
        f[ip] = fo;
    }
    return unstable;
}

template <class R, bool SH>
__device__ __forceinline__ bool collide(R (&f)[Q], R rho, R drho, const R u[3], const R F[3], const Phys<R> &ph) {
    const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const bool unstable = !(rho > R(0)) || !(usq < R(1.0 / 3.0));
    const R uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const R wp = ph.omega_p, wm = ph.omega_m;
    if constexpr (!SH) {
        {
            const R feq0 = wgt<R>(0) * rho * (R(1) + R(3) * R(0) + R(4.5) * R(0) * R(0) - R(1.5) * usq);
            const R D0 = wgt<R>(0) * (ph.A * R(0) + ph.B * (R(9) * R(0) * R(0) - R(3) * uF));
            f[0] = f[0] - wp * (R(0.5) * (f[0] + f[0]) - R(0.5) * (feq0 + feq0)) - wm * R(0) + D0;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const int ip = i + 1;
            const R cu = cdot<R>(i, u);
            const R cF = cdot<R>(i, F);
            const R wr = wgt<R>(i) * rho;
            const R fe_i = wr * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
            const R fe_o = wr * (R(1) + R(3) * (-cu) + R(4.5) * (-cu) * (-cu) - R(1.5) * usq);
            const R Bt = ph.B * (R(9) * cu * cF - R(3) * uF);
            const R Di = wgt<R>(i) * (ph.A * cF + Bt);
            const R Do = wgt<R>(i) * (Bt - ph.A * cF);
            const R fp = R(0.5) * (f[i] + f[ip]);
            const R fm = R(0.5) * (f[i] - f[ip]);
            const R ep = R(0.5) * (fe_i + fe_o);
            const R em = R(0.5) * (fe_i - fe_o);
            const R Pp = wp * (fp - ep);
            const R Pm = wm * (fm - em);
            const R fi = f[i] - Pp - Pm + Di;
            const R fo = f[ip] - Pp + Pm + Do;
            f[i] = fi;
            f[ip] = fo;
        }
    } else {
        return collide_sh<R>(f, rho, drho, u, F, ph);
    }
    return unstable;
}

// Lane helpers of the stress update: |v|, and a per-lane choice between a value and zero.
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
// v where the lane's cell sees an open face l and v > 0, else 0 (the donor-cell coefficient)
__device__ __forceinline__ float vpos_open(uint32_t m, int l, float v) {
    return (!nb_solid(m, l + 1) && v > 0.0f) ? v : 0.0f;
}
__device__ __forceinline__ float2 vpos_open(uint2 m, int l, float2 v) {
    return make_float2(vpos_open(m.x, l, v.x), vpos_open(m.y, l, v.y));
}
__device__ __forceinline__ bool lane_moving_solid(uint32_t m, int l, int) {
    return (m & MASK_MOVING) && nb_solid(m, l + 1);
}
__device__ __forceinline__ bool lane_moving_solid(uint2 m, int l, int lane) {
    return lane_moving_solid(lane == 0 ? m.x : m.y, l, 0);
}
__device__ __forceinline__ float &lane_ref(float &v, int) { return v; }
__device__ __forceinline__ float &lane_ref(float2 &v, int lane) { return lane == 0 ? v.x : v.y; }
__device__ __forceinline__ float lane_val(float v, int) { return v; }
__device__ __forceinline__ float lane_val(float2 v, int lane) { return lane == 0 ? v.x : v.y; }
template <class V>
__host__ __device__ constexpr int lanes_of() {
    return sizeof(V) / sizeof(float);
}

// Finite-volume stress update of the shifted modes in lane form (see fv_core for the
// method): V = float (one cell) or float2 (two cells), M the mask of the lane's cells.
// nb.u(l, k), nb.tau(l, c): the face-l neighbours' velocity / stress (V); nb.ub(l, lane,
// out): the boundary velocity of the solid face-l neighbour of the lane's cell.
template <class V, class M, bool VAR, class Nb>
__device__ __forceinline__ void fv_core_sh(const Phys<float> &ph, const V (&tr)[6], const V (&ur)[3], M mask,
                                           const Nb &nb, V out[6]) {
    const V half = vbc<V>(0.5f), one = vbc<V>(1.0f);
    V un[6][3];
    V G[3][3];
    // every face neighbour's u, a solid face's replaced by the mirror value 2 u_b - u(r)
    // (-u(r) at rest), so that the gradient is half the difference of the mirrored values
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = 2 * k + h;
#pragma unroll
            for (int j = 0; j < 3; ++j) un[l][j] = vsel_solid(mask, l + 1, vneg(ur[j]), nb.u(l, j));
#pragma unroll
            for (int ln = 0; ln < lanes_of<V>(); ++ln) {
                if (lane_moving_solid(mask, l, ln)) {
                    float ub[3];
                    nb.ub(l, ln, ub);
#pragma unroll
                    for (int j = 0; j < 3; ++j) lane_ref(un[l][j], ln) = __fmaf_rn(2.0f, ub[j], -lane_val(ur[j], ln));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) G[k][j] = vmul(half, vsub(un[2 * k][j], un[2 * k + 1][j]));
    }
    V net[6];
    const bool flux = !VAR || ph.flux_on;  // without VAR the flux and the source are on
    if (flux) {
        V aout, inflow[6];
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            const int k = l >> 1;
            const bool pos = (l & 1) == 0;
            // zero flux across a solid link: both coefficients zero (a solid cell's stress
            // is finite, so the inflow product adds zero)
            V ao = vpos_open(mask, l, pos ? ur[k] : vneg(ur[k]));
            V b = vpos_open(mask, l, pos ? vneg(un[l][k]) : un[l][k]);
            if constexpr (VAR) {
                if (ph.ctu_on) {
                    const int ta = k == 2 ? 0 : k + 1, tb = k == 0 ? 2 : k - 1;
                    ao = vmul(ao, vmul(vsub(one, vabs(ur[ta])), vsub(one, vabs(ur[tb]))));
                    b = vmul(b, vmul(vsub(one, vabs(un[l][ta])), vsub(one, vabs(un[l][tb]))));
                }
            }
            aout = l == 0 ? ao : vadd(aout, ao);
#pragma unroll
            for (int c = 0; c < 6; ++c) inflow[c] = l == 0 ? vmul(b, nb.tau(l, c)) : vfma(b, nb.tau(l, c), inflow[c]);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) net[c] = vfma(aout, tr[c], vneg(inflow[c]));
    }
    const bool src = !VAR || ph.src_on;
    V Sv[6];
    if (src) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int i = comp_i(c), j = comp_j(c);
            V a = vmul(tr[comp(i, 0)], G[0][j]);
            a = vfma(tr[comp(i, 1)], G[1][j], a);
            a = vfma(tr[comp(i, 2)], G[2][j], a);
            V b = vmul(tr[comp(0, j)], G[0][i]);
            b = vfma(tr[comp(1, j)], G[1][i], b);
            b = vfma(tr[comp(2, j)], G[2][i], b);
            bool fene = false;
            if constexpr (VAR) fene = ph.fene;
            if (fene) {
                // FENE-P conformation: A.grad u + (A.grad u)^T - (f A - I) / lambda
                const V fA = vrcp(vsub(one, vdiv(vadd(vadd(tr[0], tr[1]), tr[2]), vbc<V>(ph.fene_L2))));
                const V fAt = c < 3 ? vfma(fA, tr[c], vneg(one)) : vmul(fA, tr[c]);
                Sv[c] = vfma(vbc<V>(-ph.inv_l), fAt, vadd(a, b));
            } else {
                Sv[c] = vfma(vbc<V>(-ph.inv_l), tr[c], vfma(vbc<V>(ph.ep_l), vadd(G[i][j], G[j][i]), vadd(a, b)));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        V S = src ? Sv[c] : vbc<V>(0.0f);
        if constexpr (VAR) {
            if (ph.divu_on) S = vfma(tr[c], vadd(vadd(G[0][0], G[1][1]), G[2][2]), S);
            if (src && ph.gk != 0.0f) {
                const int i = comp_i(c), j = comp_j(c);
                V q = vmul(tr[comp(i, 0)], tr[comp(0, j)]);
                q = vfma(tr[comp(i, 1)], tr[comp(1, j)], q);
                q = vfma(tr[comp(i, 2)], tr[comp(2, j)], q);
                S = vfma(vbc<V>(-ph.gk), q, S);
            }
        }
        out[c] = flux ? vadd(vsub(tr[c], net[c]), S) : vadd(tr[c], S);
    }
}

// Finite-volume stress update of one fluid cell (Sec. "Discretization", "Stability
// improvements"): velocity gradient by the central-point rule (boundary velocity as the
// face value towards solid cells), donor-cell flux on the D3Q7 faces with zero flux
// across solid links, source Eq. (source) without the tau div u term, explicit Euler.
// Variants (compiled in when VAR, then chosen per solve): ph.ctu_on scales a face flux by
// the donor cell's transverse overlap (1 - |u_a|)(1 - |u_b|); ph.divu_on adds tau div u
// to the source; ph.gk != 0 adds the Giesekus term -(alpha / eta_p)(tau . tau) to it
// (with the source on).  With VAR false the method's own update is all that is compiled.
// nb.u(l, k), nb.tau(l, c): velocity / stress of the face-l neighbour (FP64 reads them
// for fluid neighbours only; the shifted modes read every face neighbour, a solid cell
// holding zero stress); nb.ub(l, out): boundary velocity of a solid face-l neighbour.
// FP64 mode keeps the face-by-face order of the plain statement; shifted modes gather
// the outflow as (sum of outgoing face velocities) * tau(r).
// fv_core's neighbour accessor seen by fv_core_sh with one lane (the lane argument of ub
// is always 0)
template <class Nb>
struct OneLaneNb {
    const Nb &n;
    __device__ __forceinline__ float u(int l, int j) const { return n.u(l, j); }
    __device__ __forceinline__ float tau(int l, int c) const { return n.tau(l, c); }
    __device__ __forceinline__ void ub(int l, int, float o[3]) const { n.ub(l, o); }
};

template <class R, bool SH, bool VAR, class Nb>
__device__ __forceinline__ void fv_core(const Phys<R> &ph, const R (&tr)[6], const R (&ur)[3], uint32_t mask,
                                        const Nb &nb, R out[6]) {
    if constexpr (SH) {
        fv_core_sh<float, uint32_t, VAR>(ph, tr, ur, mask, OneLaneNb<Nb>{nb}, out);
    } else {
        // FP64: the face-by-face order of the plain statement
        R un[6][3];
        R G[3][3];
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            if (!nb_solid(mask, l + 1)) {
#pragma unroll
                for (int j = 0; j < 3; ++j) un[l][j] = nb.u(l, j);
            } else if (mask & MASK_MOVING) {
                nb.ub(l, un[l]);
            } else {  // a resting no-slip wall
#pragma unroll
                for (int j = 0; j < 3; ++j) un[l][j] = R(0);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const bool fp_ = !nb_solid(mask, 2 * k + 1), fm_ = !nb_solid(mask, 2 * k + 2);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R up = fp_ ? R(0.5) * (ur[j] + un[2 * k][j]) : un[2 * k][j];
                const R um = fm_ ? R(0.5) * (ur[j] + un[2 * k + 1][j]) : un[2 * k + 1][j];
                G[k][j] = up - um;
            }
        }
        R net[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        // without VAR the flux and the source are on (a solve with either off takes the VAR build)
        if (!VAR || ph.flux_on) {
#pragma unroll
            for (int l = 0; l < 6; ++l) {
                const int k = l >> 1;
                const int s = (l & 1) ? -1 : 1;
                if (nb_solid(mask, l + 1)) continue;
                const R vout = s > 0 ? ur[k] : -ur[k];
                const R vin = s > 0 ? -un[l][k] : un[l][k];
                R tout = R(1), tin = R(1);
                if (VAR && ph.ctu_on) {
                    const int ta = k == 2 ? 0 : k + 1, tb = k == 0 ? 2 : k - 1;
                    tout = (R(1) - fabs(ur[ta])) * (R(1) - fabs(ur[tb]));
                    tin = (R(1) - fabs(un[l][ta])) * (R(1) - fabs(un[l][tb]));
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const R Jo = vout > R(0) ? (vout * tout) * tr[c] : R(0);
                    const R Ji = vin > R(0) ? (vin * tin) * nb.tau(l, c) : R(0);
                    net[c] = net[c] + (Jo - Ji);
                }
            }
        }
        R Sv[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        if (!VAR || ph.src_on) {  // one test for all six components
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const int i = comp_i(c), j = comp_j(c);
                R a = R(0), b = R(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) a = a + tr[comp(i, k)] * G[k][j];
#pragma unroll
                for (int k = 0; k < 3; ++k) b = b + tr[comp(k, j)] * G[k][i];
                if (VAR && ph.fene) {
                    // FENE-P conformation: A.grad u + (A.grad u)^T - (f A - I) / lambda
                    const R fA = fene_factor<R>(ph, tr[0], tr[1], tr[2]);
                    Sv[c] = a + b - ph.inv_l * (c < 3 ? fA * tr[c] - R(1) : fA * tr[c]);
                } else {
                    Sv[c] = a + b + ph.ep_l * (G[i][j] + G[j][i]) - ph.inv_l * tr[c];
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            R S = Sv[c];
            if (VAR && ph.divu_on) S = S + tr[c] * ((G[0][0] + G[1][1]) + G[2][2]);
            if (VAR && ph.src_on && ph.gk != R(0)) {
                const int i = comp_i(c), j = comp_j(c);
                R q = R(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) q = q + tr[comp(i, k)] * tr[comp(k, j)];
                S = S - ph.gk * q;
            }
            out[c] = tr[c] - net[c] + S;
        }
    }
}

} // namespace lbve

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

#include "lbve_device.cuh"
#include "lbve_launch.h"

namespace lbve {

template <class S>
struct KArgs {
    using R = typename Store<S>::R;
    Geo g;
    Phys<R> ph;
    S *f;
    const R *tau;   // tau^t
    R *tau_out;     // tau^{t+1}
    R *u;           // u^t (written by k_lb, read by k_fv)
    const uint8_t *flag;
    const PartDev *parts;
};

// Load f_i^t of cell r from its AA location for the given parity.
template <class S, int PAR>
__device__ __forceinline__ void load_pdfs(const KArgs<S> &a, const Cell &cl, long long r,
                                          typename Store<S>::R (&f)[Q]) {
    using R = typename Store<S>::R;
    const long long np = a.g.np;
    const R inv = a.ph.inv_scale;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S *p = PAR == 0 ? a.f + (long long)i * np + r
                              : a.f + (long long)copp(i) * np + cl.idx(-cx(i), -cy(i), -cz(i));
        f[i] = Store<S>::ld(p, inv);
    }
}

// Store post-collision f*_i with AA addressing; links into solid cells bounce back with
// the moving-wall term of Eq. (ubb): f_-i(r, t+1) = f*_i(r) - 6 w_i rho c_i . u_b.
template <class S, int PAR>
__device__ __forceinline__ void store_pdfs(const KArgs<S> &a, const Cell &cl, long long r,
                                           const typename Store<S>::R (&fs)[Q], typename Store<S>::R rho) {
    using R = typename Store<S>::R;
    const long long np = a.g.np;
    const R sc = a.ph.scale;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (i == 0) {
            Store<S>::st(a.f + r, fs[0], sc);
            continue;
        }
        const long long nb = cl.idx(cx(i), cy(i), cz(i));
        const int fl = a.flag[nb];
        if (fl == FLAG_FLUID) {
            S *p = PAR == 0 ? a.f + (long long)copp(i) * np + r : a.f + (long long)i * np + nb;
            Store<S>::st(p, fs[i], sc);
        } else {
            R X = R(0);
            if (fl != FLAG_NOSLIP) {
                R ub[3];
                boundary_velocity<R>(a.g, a.ph, a.parts, fl, cl.X(cx(i)), cl.Y(cy(i)), cl.Z(cz(i)), ub);
                X = R(6) * wgt<R>(i) * rho * cdot<R>(i, ub);
            }
            S *p = PAR == 0 ? a.f + (long long)i * np + nb : a.f + (long long)copp(i) * np + r;
            Store<S>::st(p, fs[i] - X, sc);
        }
    }
}

// LB half of the step for one fluid cell: F = g + F^p(tau^t), moments, u^t written out,
// TRT collision with forcing, AA streaming with bounce-back.
template <class S, int PAR>
__device__ __forceinline__ void lb_cell(const KArgs<S> &a, const Cell &cl, long long r) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, cl, r, a.tau, a.flag, Fp);
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = a.ph.g[k] + Fp[k];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
#pragma unroll
    for (int k = 0; k < 3; ++k) a.u[k * a.g.np + r] = u[k];
    collide<R, SH>(f, rho, drho, u, F, a.ph);
    store_pdfs<S, PAR>(a, cl, r, f, rho);
}

template <class S, int PAR>
__global__ void __launch_bounds__(256) k_lb(KArgs<S> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.nx) return;
    const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
    const long long r = cl.self();
    if (a.flag[r] != FLAG_FLUID) return;
    lb_cell<S, PAR>(a, cl, r);
}

template <class S>
__global__ void __launch_bounds__(256) k_fv(KArgs<S> a) {
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.nx) return;
    const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
    const long long r = cl.self();
    R out[6];
    if (a.flag[r] != FLAG_FLUID) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.tau_out[c * a.g.np + r] = R(0);
        return;
    }
    fv_cell<R>(a.g, a.ph, cl, r, a.tau, a.u, a.flag, a.parts, out);
#pragma unroll
    for (int c = 0; c < 6; ++c) a.tau_out[c * a.g.np + r] = out[c];
}

// ---------------------------------------------------------------------------------
// momentum exchange (Sec. "Moving boundaries"): for every link (fluid cell r,
// direction i into a tracked solid cell) the force c_i (2 f*_i - 6 w_i rho c_i.u_b) and
// its torque about the owning particle.  Runs before k_lb on the same f^t and repeats
// the cell's collision, so f*_i is exactly the value k_lb streams.
// ---------------------------------------------------------------------------------
template <class S, int PAR>
__global__ void __launch_bounds__(128) k_momentum_exchange(KArgs<S> a, const long long *__restrict__ links, int nlinks,
                                                           double *__restrict__ contrib) {
    using R = typename Store<S>::R;
    constexpr bool SH = Store<S>::shifted;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    const long long code = links[l];
    const int i = (int)(code & 31);
    const long long r = code >> 5;
    const int x = (int)(r % a.g.nx), y = (int)((r / a.g.nx) % a.g.ny), z = (int)(r / ((long long)a.g.nx * a.g.ny));
    const Cell cl(a.g, x, y, z);
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, cl, r, a.tau, a.flag, Fp);
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = a.ph.g[k] + Fp[k];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    collide<R, SH>(f, rho, drho, u, F, a.ph);
    // f*_i as a full population (the stored deviation plus w_i rho0 in shifted modes)
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
    R wi = i < 7 ? wgt<R>(1) : wgt<R>(7);
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
    double *o = contrib + (long long)l * 8;
    o[0] = Fl[0];
    o[1] = Fl[1];
    o[2] = Fl[2];
    o[3] = T[0];
    o[4] = T[1];
    o[5] = T[2];
    o[6] = (double)fl;
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
    for (int c = 0; c < 6; ++c) tau_dst[c * a.g.np + r] = tau_in ? (R)tau_in[c * ld + k] : R(0);
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
    const long long r = cl.self();
    const long long k = r - (long long)z0 * a.g.nx * a.g.ny;
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
    polymer_force<R>(a.g, cl, r, a.tau, a.flag, Fp);
#pragma unroll
    for (int j = 0; j < 3; ++j) F[j] = a.ph.g[j] + Fp[j];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    if (rho_out) rho_out[k] = SH ? (double)a.ph.rho0 + (double)drho : (double)rho;
    for (int j = 0; j < 3; ++j)
        if (u_out) u_out[j * ld + k] = (double)u[j];
    for (int c = 0; c < 6; ++c)
        if (tau_out) tau_out[c * ld + k] = (double)a.tau[c * a.g.np + r];
}

// PDFs of every cell to / from unshifted FP64 in the plain (pre-collision) layout.
template <class S, int PAR>
__global__ void k_pdfs_io(KArgs<S> a, double *__restrict__ io, int write) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.g.nx) return;
    const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
    const long long r = cl.self();
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
    const long long r = cells[k];
    const int x = (int)(r % a.g.nx), y = (int)((r / a.g.nx) % a.g.ny), z = (int)(r / ((long long)a.g.nx * a.g.ny));
    const Cell cl(a.g, x, y, z);
    R f[Q];
    load_pdfs<S, PAR>(a, cl, r, f);
    double *o = out + (long long)k * 29;
    for (int i = 0; i < Q; ++i) o[i] = (double)f[i] + (SH ? wgt<double>(i) * (double)a.ph.rho0 : 0.0);
    for (int j = 19; j < 29; ++j) o[j] = 0.0;
    if (a.flag[r] != FLAG_FLUID) return;
    R Fp[3], F[3], u[3], rho, drho;
    polymer_force<R>(a.g, cl, r, a.tau, a.flag, Fp);
    for (int j = 0; j < 3; ++j) F[j] = a.ph.g[j] + Fp[j];
    moments<R, SH>(f, F, a.ph.rho0, rho, drho, u);
    o[19] = SH ? (double)a.ph.rho0 + (double)drho : (double)rho;
    for (int j = 0; j < 3; ++j) o[20 + j] = (double)u[j];
    for (int c = 0; c < 6; ++c) o[23 + c] = (double)a.tau[c * a.g.np + r];
}

// Per-block FP64 partial sums over fluid cells: mass, momentum, count, bad-value flag.
template <class S, int PAR>
__global__ void __launch_bounds__(256) k_reduce(KArgs<S> a, double *__restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (x < a.g.nx) {
        const Cell cl(a.g, x, blockIdx.y, blockIdx.z);
        const long long r = cl.self();
        if (a.flag[r] == FLAG_FLUID) {
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

} // namespace lbve

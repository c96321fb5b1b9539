// lbve2d.cu -- the two-dimensional coupled step (include/lbve2d.h): D2Q9 TRT lattice
// Boltzmann with Guo forcing and a D2Q5 finite-volume Oldroyd-B stress update (Kuron et
// al., arXiv:2009.12279, Sec. "Lid-driven cavity", Sec. "Four-roll mill").
//
// Two kernels per step: k2_lb (polymer force, moments, collision, push streaming with
// bounce-back into the second PDF array; writes u) and k2_fv (stress update from tau^t
// and u^t).  The 2-D cases of the paper are small (194^2, 214^2 cells), so the PDFs use
// two arrays and plain per-cell kernels.  FP64 storage keeps f_i and evaluates every
// formula in the operation order of its plain statement (this unit is built with FMA
// contraction off); FP32 storage keeps the deviation f_i - w_i rho0 and forms the TRT
// non-equilibrium parts before scaling them by rounded constants, as the 3-D kernels do.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbve2d.h"

namespace {

constexpr int Q2 = 9;
__host__ __device__ constexpr int c2x(int i) { return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr int c2y(int i) { return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int opp2(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <class R>
__host__ __device__ constexpr R w2(int i) {
    return i == 0 ? R(4.0 / 9.0) : (i < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}
// stress layout xx, yy, xy
__host__ __device__ constexpr int cmp2(int a, int b) { return a == b ? a : 2; }

template <class R>
struct Phys2 {
    R omega_p, omega_m, A, B, ep_l, inv_l;
    R g[2];
    R rho0;  // shift base of the stored deviations (0 in FP64 mode)
    int flux_on, src_on;
};

template <class R>
struct Args2 {
    int nx, ny, per[2];
    long long n;
    Phys2<R> ph;
    const R *f_in;
    R *f_out;
    const R *tau;
    R *tau_out;
    const R *u_in;
    R *u_out;
    const uint8_t *flag;
    const R *ub;     // 2n: velocity of solid cells
    const R *force;  // 2n or nullptr
};

// neighbour index (periodic wrap), -1 outside a closed side
template <class R>
__device__ __forceinline__ long long nb2(const Args2<R> &a, int x, int y, int dx, int dy) {
    int qx = x + dx, qy = y + dy;
    if (qx < 0 || qx >= a.nx) {
        if (!a.per[0]) return -1;
        qx = (qx + a.nx) % a.nx;
    }
    if (qy < 0 || qy >= a.ny) {
        if (!a.per[1]) return -1;
        qy = (qy + a.ny) % a.ny;
    }
    return (long long)qx + (long long)a.nx * qy;
}

template <class R>
__device__ __forceinline__ bool fluid2(const Args2<R> &a, long long r) { return r >= 0 && a.flag[r] == 0; }

template <class R>
__device__ __forceinline__ R cvec(int i, R v0, R v1) {
    // c_i . v for components in {-1, 0, 1}, accumulated as the plain sum c_x v_x + c_y v_y
    const int cx = c2x(i), cy = c2y(i);
    R t = cx == 0 ? R(0) : (cx > 0 ? v0 : -v0);
    if (cy != 0) t = cx == 0 ? (cy > 0 ? v1 : -v1) : (cy > 0 ? t + v1 : t - v1);
    return t;
}

// Polymer force, Eq. (force) on the D2Q5 faces +x, -x, +y, -y.
template <class R>
__device__ __forceinline__ void polymer_force2(const Args2<R> &a, int x, int y, long long r, R Fp[2]) {
    Fp[0] = R(0);
    Fp[1] = R(0);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int k = l >> 1, s = (l & 1) ? -1 : 1;
        const long long nb = nb2(a, x, y, k == 0 ? s : 0, k == 1 ? s : 0);
        const bool fl = fluid2(a, nb);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = cmp2(k, j);
            const R tr = a.tau[c * a.n + r];
            const R tf = fl ? R(0.5) * (tr + a.tau[c * a.n + nb]) : tr;
            Fp[j] = s > 0 ? Fp[j] + tf : Fp[j] - tf;
        }
    }
}

// F = (g + F_field) + F^p and the moments of Eq. (macroscopic-velocity).
template <class R, bool SH>
__device__ __forceinline__ void macro2(const Args2<R> &a, int x, int y, long long r, const R (&f)[Q2], R F[2], R &rho,
                                       R &drho, R u[2]) {
    R Fp[2];
    polymer_force2(a, x, y, r, Fp);
#pragma unroll
    for (int j = 0; j < 2; ++j) F[j] = (a.ph.g[j] + (a.force ? a.force[j * a.n + r] : R(0))) + Fp[j];
    if constexpr (!SH) {
        R s = R(0), jx = R(0), jy = R(0);
#pragma unroll
        for (int i = 0; i < Q2; ++i) s = s + f[i];
        // sum over i of f_i c_i in direction order
        jx = ((((jx + f[1]) - f[2]) + f[5]) - f[6]) + f[7];
        jx = jx - f[8];
        jy = ((((jy + f[3]) - f[4]) + f[5]) - f[6]) - f[7];
        jy = jy + f[8];
        rho = s;
        drho = s;
        u[0] = (jx + R(0.5) * F[0]) / s;
        u[1] = (jy + R(0.5) * F[1]) / s;
    } else {
        drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        rho = a.ph.rho0 + drho;
        const R jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[7] - f[8]);
        const R jy = (f[3] - f[4]) + (f[5] - f[6]) + (f[8] - f[7]);
        const R ir = R(1) / rho;
        u[0] = (jx + R(0.5) * F[0]) * ir;
        u[1] = (jy + R(0.5) * F[1]) * ir;
    }
}

template <class R, bool SH>
__global__ void __launch_bounds__(128) k2_lb(Args2<R> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long r = (long long)x + (long long)a.nx * y;
    if (a.flag[r] != 0) return;
    R f[Q2];
#pragma unroll
    for (int i = 0; i < Q2; ++i) f[i] = a.f_in[i * a.n + r];
    R F[2], rho, drho, u[2];
    macro2<R, SH>(a, x, y, r, f, F, rho, drho, u);
    a.u_out[r] = u[0];
    a.u_out[a.n + r] = u[1];
    const R wp = a.ph.omega_p, wm = a.ph.omega_m;
    const R usq = u[0] * u[0] + u[1] * u[1];
    const R uF = u[0] * F[0] + u[1] * F[1];
    R fs[Q2];
    if constexpr (!SH) {
        // Eqs. (lb), (lb-equilibrium), (guo) as plainly stated, population by population
        R feq[Q2], D[Q2];
#pragma unroll
        for (int i = 0; i < Q2; ++i) {
            const R cu = cvec<R>(i, u[0], u[1]);
            const R cF = cvec<R>(i, F[0], F[1]);
            feq[i] = w2<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
            D[i] = w2<R>(i) * (a.ph.A * cF + a.ph.B * (R(9) * cu * cF - R(3) * uF));
        }
#pragma unroll
        for (int i = 0; i < Q2; ++i) {
            const int ip = opp2(i);
            const R fp = R(0.5) * (f[i] + f[ip]), fm = R(0.5) * (f[i] - f[ip]);
            const R ep = R(0.5) * (feq[i] + feq[ip]), em = R(0.5) * (feq[i] - feq[ip]);
            fs[i] = f[i] - wp * (fp - ep) - wm * (fm - em) + D[i];
        }
    } else {
        // deviations; per pair (i, -i) with k = 1/(6 w_i), k2 = 1/(2 w_i) exactly
        // representable (1.5, 4.5 for w = 1/9; 6, 18 for w = 1/36), the non-equilibrium
        // parts k (f_i - f_-i) - rho c.u and k2 (f_i + f_-i) - e_sym are formed with one
        // rounding and only then scaled by the rounded rates
        const R q = R(1.5) * usq, u3F = R(3) * uF;
        fs[0] = f[0] - wp * (f[0] - w2<R>(0) * (drho - rho * q)) - w2<R>(0) * a.ph.B * u3F;
#pragma unroll
        for (int i = 1; i < Q2; i += 2) {
            const int ip = i + 1;
            const bool axis = i < 5;
            const R k = axis ? R(1.5) : R(6), k2 = axis ? R(4.5) : R(18);
            const R cu = cvec<R>(i, u[0], u[1]);
            const R cF = cvec<R>(i, F[0], F[1]);
            const R esym = drho + rho * (R(4.5) * cu * cu - q);
            const R nsym = __fmaf_rn(k2, f[i] + f[ip], -esym);
            const R nanti = __fmaf_rn(k, f[i] - f[ip], -(rho * cu));
            const R P = (R(0.5) * wp / k2) * nsym - (w2<R>(i) * a.ph.B) * (R(9) * cu * cF - u3F);
            const R M = (R(0.5) * wm / k) * nanti - (w2<R>(i) * a.ph.A) * cF;
            fs[i] = f[i] - P - M;
            fs[ip] = f[ip] - P + M;
        }
    }
    // push streaming with bounce-back, Eq. (ubb)
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
        const long long nb = nb2(a, x, y, c2x(i), c2y(i));
        if (fluid2(a, nb)) {
            a.f_out[i * a.n + nb] = fs[i];
        } else {
            R cub = R(0);
            if (nb >= 0) cub = cvec<R>(i, a.ub[nb], a.ub[a.n + nb]);
            a.f_out[opp2(i) * a.n + r] = fs[i] - R(6) * w2<R>(i) * rho * cub;
        }
    }
}

// Eqs. (continuity)-(source) on the D2Q5 faces, explicit Euler.
template <class R, bool SH>
__global__ void __launch_bounds__(128) k2_fv(Args2<R> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long r = (long long)x + (long long)a.nx * y;
    if (a.flag[r] != 0) {
        for (int c = 0; c < 3; ++c) a.tau_out[c * a.n + r] = R(0);
        return;
    }
    R tr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) tr[c] = a.tau[c * a.n + r];
    R G[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const long long np_ = nb2(a, x, y, k == 0 ? 1 : 0, k == 1 ? 1 : 0);
        const long long nm_ = nb2(a, x, y, k == 0 ? -1 : 0, k == 1 ? -1 : 0);
        const bool fp_ = fluid2(a, np_), fm_ = fluid2(a, nm_);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const R ur = a.u_in[j * a.n + r];
            const R ubp = np_ >= 0 ? a.ub[j * a.n + np_] : R(0);
            const R ubm = nm_ >= 0 ? a.ub[j * a.n + nm_] : R(0);
            const R up = fp_ ? R(0.5) * (ur + a.u_in[j * a.n + np_]) : ubp;
            const R um = fm_ ? R(0.5) * (ur + a.u_in[j * a.n + nm_]) : ubm;
            G[k][j] = up - um;
        }
    }
    R net[3] = {R(0), R(0), R(0)};
    if (a.ph.flux_on) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int k = l >> 1, s = (l & 1) ? -1 : 1;
            const long long nb = nb2(a, x, y, k == 0 ? s : 0, k == 1 ? s : 0);
            if (!fluid2(a, nb)) continue;
            const R uk = a.u_in[k * a.n + r], unk = a.u_in[k * a.n + nb];
            const R vout = s > 0 ? uk : -uk;
            const R vin = s > 0 ? -unk : unk;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const R Jo = vout > R(0) ? vout * tr[c] : R(0);
                const R Ji = vin > R(0) ? vin * a.tau[c * a.n + nb] : R(0);
                net[c] = net[c] + (Jo - Ji);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R S = R(0);
        if (a.ph.src_on) {
            const int i = c == 1 ? 1 : 0, j = c == 0 ? 0 : 1;
            R p = R(0), q = R(0);
#pragma unroll
            for (int k = 0; k < 2; ++k) p = p + tr[cmp2(i, k)] * G[k][j];
#pragma unroll
            for (int k = 0; k < 2; ++k) q = q + tr[cmp2(k, j)] * G[k][i];
            S = p + q + a.ph.ep_l * (G[i][j] + G[j][i]) - a.ph.inv_l * tr[c];
        }
        a.tau_out[c * a.n + r] = tr[c] - net[c] + S;
    }
}

template <class R, bool SH>
__global__ void k2_init(Args2<R> a, R *f, R *tau, const double *rho_in, const double *u_in, const double *tau_in,
                        double rho_ref) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    const double rho = rho_in ? rho_in[r] : rho_ref;
    const double u0 = u_in ? u_in[r] : 0.0, u1 = u_in ? u_in[a.n + r] : 0.0;
    const double usq = u0 * u0 + u1 * u1;
    for (int i = 0; i < Q2; ++i) {
        const double cu = cvec<double>(i, u0, u1);
        double v;
        if constexpr (!SH)
            v = w2<double>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
        else
            v = w2<double>(i) * ((rho - (double)a.ph.rho0) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
        f[i * a.n + r] = (R)v;
    }
    for (int c = 0; c < 3; ++c) tau[c * a.n + r] = tau_in ? (R)tau_in[c * a.n + r] : R(0);
}

template <class R, bool SH>
__global__ void k2_read(Args2<R> a, double *rho_out, double *u_out, double *tau_out, double *f_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long r = (long long)x + (long long)a.nx * y;
    R f[Q2];
#pragma unroll
    for (int i = 0; i < Q2; ++i) f[i] = a.f_in[i * a.n + r];
    if (f_out)
        for (int i = 0; i < Q2; ++i) f_out[i * a.n + r] = (double)f[i] + (SH ? w2<double>(i) * (double)a.ph.rho0 : 0.0);
    const bool fl = a.flag[r] == 0;
    R F[2], rho = R(0), drho = R(0), u[2] = {R(0), R(0)};
    if (fl) macro2<R, SH>(a, x, y, r, f, F, rho, drho, u);
    if (rho_out) rho_out[r] = fl ? (SH ? (double)a.ph.rho0 + (double)drho : (double)rho) : 0.0;
    if (u_out)
        for (int j = 0; j < 2; ++j) u_out[j * a.n + r] = fl ? (double)u[j] : 0.0;
    if (tau_out)
        for (int c = 0; c < 3; ++c) tau_out[c * a.n + r] = fl ? (double)a.tau[c * a.n + r] : 0.0;
}

} // namespace

struct lbve2d_ctx {
    lbve2d_params p;
    cudaStream_t stream = nullptr;
    long long n = 0, t = 0;
    int cur = 0;  // f[cur], tau[cur] hold the state at time t
    size_t rb = 8;
    void *f[2] = {nullptr, nullptr}, *tau[2] = {nullptr, nullptr}, *u = nullptr, *ub = nullptr, *force = nullptr;
    uint8_t *flag = nullptr;
    double *stage = nullptr;  // FP64 staging, 10 n doubles
    Phys2<double> ph;
    std::string err;
};

namespace {
std::string g_err2;

lbve_status fail2(lbve2d_ctx *c, lbve_status s, const std::string &m) {
    (c ? c->err : g_err2) = m;
    return s;
}
lbve_status cuda2(lbve2d_ctx *c, cudaError_t e, const char *where) {
    return fail2(c, LBVE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK2(expr, where)                                   \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda2(c, e_, where); \
    } while (0)

bool valid2(const lbve2d_params *p, std::string &why) {
    if (!p) return why = "params is NULL", false;
    if (p->nx < 1 || p->ny < 1 || p->ny > 65535) return why = "grid dimensions out of range", false;
    if ((long long)p->nx * p->ny > (1LL << 31) - 1) return why = "grid too large", false;
    if (!(p->eta > 0.0) || !(p->beta >= 0.0 && p->beta < 1.0) || !(p->rho0 > 0.0))
        return why = "eta > 0, beta in [0, 1) and rho0 > 0 are required", false;
    if (p->beta > 0.0 && !(p->lambda_p > 0.0)) return why = "lambda_p must be > 0 when beta > 0", false;
    if (p->pdf_prec != LBVE_F64 && p->pdf_prec != LBVE_F32) return why = "pdf_prec must be LBVE_F64 or LBVE_F32", false;
    if (p->fv_terms < 0 || p->fv_terms > 3) return why = "fv_terms must use the FLUX and SOURCE bits only", false;
    if (!(p->magic >= 0.0)) return why = "magic must be >= 0", false;
    return true;
}

template <class R>
Args2<R> args2(const lbve2d_ctx *c) {
    Args2<R> a;
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.per[0] = c->p.periodic[0] ? 1 : 0;
    a.per[1] = c->p.periodic[1] ? 1 : 0;
    a.n = c->n;
    a.ph.omega_p = (R)c->ph.omega_p;
    a.ph.omega_m = (R)c->ph.omega_m;
    a.ph.A = (R)c->ph.A;
    a.ph.B = (R)c->ph.B;
    a.ph.ep_l = (R)c->ph.ep_l;
    a.ph.inv_l = (R)c->ph.inv_l;
    a.ph.g[0] = (R)c->ph.g[0];
    a.ph.g[1] = (R)c->ph.g[1];
    a.ph.rho0 = (R)c->ph.rho0;
    a.ph.flux_on = c->ph.flux_on;
    a.ph.src_on = c->ph.src_on;
    a.f_in = (const R *)c->f[c->cur];
    a.f_out = (R *)c->f[c->cur ^ 1];
    a.tau = (const R *)c->tau[c->cur];
    a.tau_out = (R *)c->tau[c->cur ^ 1];
    a.u_in = (const R *)c->u;
    a.u_out = (R *)c->u;
    a.flag = c->flag;
    a.ub = (const R *)c->ub;
    a.force = (const R *)c->force;
    return a;
}

dim3 block2d() { return dim3(64, 2); }
dim3 grid2d(const lbve2d_ctx *c) { return dim3((unsigned)((c->p.nx + 63) / 64), (unsigned)((c->p.ny + 1) / 2)); }

template <class R, bool SH>
cudaError_t step_impl(lbve2d_ctx *c) {
    Args2<R> a = args2<R>(c);
    k2_lb<R, SH><<<grid2d(c), block2d(), 0, c->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k2_fv<R, SH><<<grid2d(c), block2d(), 0, c->stream>>>(a);
    return cudaGetLastError();
}

// host FP64 field (2n) -> device field of the storage real type
lbve_status upload_real(lbve2d_ctx *c, void *dst, const double *src, long long count) {
    if (c->rb == 8) {
        CK2(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream), "upload");
    } else {
        std::vector<float> h((size_t)count);
        for (long long k = 0; k < count; ++k) h[k] = (float)src[k];
        CK2(cudaMemcpyAsync(dst, h.data(), sizeof(float) * count, cudaMemcpyHostToDevice, c->stream), "upload");
        CK2(cudaStreamSynchronize(c->stream), "upload sync");
    }
    return LBVE_OK;
}

} // namespace

extern "C" {

void lbve2d_default_params(lbve2d_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = 32;
    p->periodic[0] = p->periodic[1] = 1;
    p->eta = 1.0 / 6.0;
    p->beta = 0.5;
    p->lambda_p = 1000.0;
    p->rho0 = 1.0;
    p->magic = 3.0 / 16.0;
    p->pdf_prec = LBVE_F32;
    p->fv_terms = LBVE_FV_FLUX | LBVE_FV_SOURCE;
}

lbve_status lbve2d_create(const lbve2d_params *p, void *cuda_stream, lbve2d_ctx **out) {
    if (!out) return LBVE_EINVAL;
    *out = nullptr;
    std::string why;
    if (!valid2(p, why)) return fail2(nullptr, LBVE_EINVAL, why);
    lbve2d_ctx *c = new (std::nothrow) lbve2d_ctx();
    if (!c) return LBVE_ENOMEM;
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    c->n = (long long)p->nx * p->ny;
    c->rb = p->pdf_prec == LBVE_F64 ? 8 : 4;
    // TRT rates from the viscosity and the magic product (Sec. "Lattice Boltzmann")
    Phys2<double> &ph = c->ph;
    std::memset(&ph, 0, sizeof(ph));
    const double nu_n = (1.0 - p->beta) * p->eta / p->rho0;
    const double magic = p->magic > 0.0 ? p->magic : 3.0 / 16.0;
    ph.omega_p = 1.0 / (3.0 * nu_n + 0.5);
    const double tp = 1.0 / ph.omega_p - 0.5;
    ph.omega_m = 1.0 / (magic / tp + 0.5);
    ph.A = 3.0 * (1.0 - 0.5 * ph.omega_m);
    ph.B = 1.0 - 0.5 * ph.omega_p;
    const double eta_p = p->beta * p->eta;
    ph.ep_l = p->beta > 0.0 ? eta_p / p->lambda_p : 0.0;
    ph.inv_l = p->lambda_p > 0.0 ? 1.0 / p->lambda_p : 0.0;
    ph.g[0] = p->body_force[0];
    ph.g[1] = p->body_force[1];
    ph.rho0 = p->pdf_prec == LBVE_F64 ? 0.0 : p->rho0;
    const int terms = (p->fv_terms & 3) == 0 ? 3 : p->fv_terms;
    ph.flux_on = (terms & LBVE_FV_FLUX) != 0;
    ph.src_on = (terms & LBVE_FV_SOURCE) != 0;
    const size_t n = (size_t)c->n;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&c->f[k], Q2 * n * c->rb);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&c->tau[k], 3 * n * c->rb);
    if (e == cudaSuccess) e = cudaMalloc(&c->u, 2 * n * c->rb);
    if (e == cudaSuccess) e = cudaMalloc(&c->ub, 2 * n * c->rb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->flag, n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->stage, 15 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, n, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ub, 0, 2 * n * c->rb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->u, 0, 2 * n * c->rb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->tau[1], 0, 3 * n * c->rb, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_err2 = std::string("device set-up failed: ") + cudaGetErrorString(e);
        lbve2d_destroy(c);
        return e == cudaErrorMemoryAllocation ? LBVE_ENOMEM : LBVE_ECUDA;
    }
    lbve_status s = lbve2d_init_fields(c, nullptr, nullptr, nullptr);
    if (s != LBVE_OK) {
        g_err2 = c->err;
        lbve2d_destroy(c);
        return s;
    }
    *out = c;
    return LBVE_OK;
}

lbve_status lbve2d_destroy(lbve2d_ctx *c) {
    if (!c) return LBVE_EINVAL;
    cudaStreamSynchronize(c->stream);
    for (void *p : {c->f[0], c->f[1], c->tau[0], c->tau[1], c->u, c->ub, c->force, (void *)c->flag, (void *)c->stage})
        if (p) cudaFree(p);
    delete c;
    return LBVE_OK;
}

lbve_status lbve2d_set_geometry(lbve2d_ctx *c, const uint8_t *flags, const double *ub) {
    if (!c) return LBVE_EINVAL;
    if (!flags) return fail2(c, LBVE_EINVAL, "flags is NULL");
    const int nx = c->p.nx, ny = c->p.ny;
    for (long long r = 0; r < c->n; ++r) {
        if (flags[r] != 0) continue;
        const int x = (int)(r % nx), y = (int)(r / nx);
        if ((!c->p.periodic[0] && (x == 0 || x == nx - 1)) || (!c->p.periodic[1] && (y == 0 || y == ny - 1)))
            return fail2(c, LBVE_EINVAL, "fluid cell in the outer layer of a non-periodic direction");
    }
    CK2(cudaMemcpyAsync(c->flag, flags, (size_t)c->n, cudaMemcpyHostToDevice, c->stream), "upload flags");
    if (ub) {
        lbve_status s = upload_real(c, c->ub, ub, 2 * c->n);
        if (s != LBVE_OK) return s;
    } else {
        CK2(cudaMemsetAsync(c->ub, 0, 2 * (size_t)c->n * c->rb, c->stream), "clear ub");
    }
    CK2(cudaStreamSynchronize(c->stream), "geometry sync");
    return LBVE_OK;
}

lbve_status lbve2d_set_force_field(lbve2d_ctx *c, const double *F) {
    if (!c) return LBVE_EINVAL;
    if (!F) {
        CK2(cudaStreamSynchronize(c->stream), "force sync");
        if (c->force) cudaFree(c->force);
        c->force = nullptr;
        return LBVE_OK;
    }
    if (!c->force) CK2(cudaMalloc(&c->force, 2 * (size_t)c->n * c->rb), "force allocation");
    lbve_status s = upload_real(c, c->force, F, 2 * c->n);
    if (s != LBVE_OK) return s;
    CK2(cudaStreamSynchronize(c->stream), "force sync");
    return LBVE_OK;
}

lbve_status lbve2d_init_fields(lbve2d_ctx *c, const double *rho, const double *u, const double *tau) {
    if (!c) return LBVE_EINVAL;
    const long long n = c->n;
    double *srho = c->stage, *su = c->stage + n, *stau = c->stage + 3 * n;
    if (rho) CK2(cudaMemcpyAsync(srho, rho, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "init copy");
    if (u) CK2(cudaMemcpyAsync(su, u, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, c->stream), "init copy");
    if (tau) CK2(cudaMemcpyAsync(stau, tau, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream), "init copy");
    c->cur = 0;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (c->rb == 8) {
        Args2<double> a = args2<double>(c);
        k2_init<double, false><<<nb, 256, 0, c->stream>>>(a, (double *)c->f[0], (double *)c->tau[0], rho ? srho : nullptr,
                                                          u ? su : nullptr, tau ? stau : nullptr, c->p.rho0);
    } else {
        Args2<float> a = args2<float>(c);
        k2_init<float, true><<<nb, 256, 0, c->stream>>>(a, (float *)c->f[0], (float *)c->tau[0], rho ? srho : nullptr,
                                                        u ? su : nullptr, tau ? stau : nullptr, c->p.rho0);
    }
    CK2(cudaGetLastError(), "init kernel");
    CK2(cudaStreamSynchronize(c->stream), "init sync");
    c->t = 0;
    return LBVE_OK;
}

lbve_status lbve2d_step(lbve2d_ctx *c, int nsteps) {
    if (!c) return LBVE_EINVAL;
    if (nsteps < 0) return fail2(c, LBVE_EINVAL, "nsteps must be >= 0");
    for (int k = 0; k < nsteps; ++k) {
        const cudaError_t e = c->rb == 8 ? step_impl<double, false>(c) : step_impl<float, true>(c);
        CK2(e, "step kernels");
        c->cur ^= 1;
        c->t++;
    }
    return LBVE_OK;
}

static lbve_status read_impl(lbve2d_ctx *c, double *rho, double *u, double *tau, double *f) {
    const long long n = c->n;
    double *drho = c->stage, *du = c->stage + n, *dtau = c->stage + 3 * n, *df = c->stage + 6 * n;
    if (c->rb == 8) {
        Args2<double> a = args2<double>(c);
        k2_read<double, false><<<grid2d(c), block2d(), 0, c->stream>>>(a, drho, du, dtau, f ? df : nullptr);
    } else {
        Args2<float> a = args2<float>(c);
        k2_read<float, true><<<grid2d(c), block2d(), 0, c->stream>>>(a, drho, du, dtau, f ? df : nullptr);
    }
    CK2(cudaGetLastError(), "read kernel");
    if (rho) CK2(cudaMemcpyAsync(rho, drho, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "read copy");
    if (u) CK2(cudaMemcpyAsync(u, du, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->stream), "read copy");
    if (tau) CK2(cudaMemcpyAsync(tau, dtau, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream), "read copy");
    if (f) CK2(cudaMemcpyAsync(f, df, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, c->stream), "read copy");
    CK2(cudaStreamSynchronize(c->stream), "read sync");
    return LBVE_OK;
}

lbve_status lbve2d_read_fields(lbve2d_ctx *c, double *rho, double *u, double *tau) {
    if (!c) return LBVE_EINVAL;
    return read_impl(c, rho, u, tau, nullptr);
}

lbve_status lbve2d_read_pdfs(lbve2d_ctx *c, double *f) {
    if (!c) return LBVE_EINVAL;
    if (!f) return fail2(c, LBVE_EINVAL, "f is NULL");
    return read_impl(c, nullptr, nullptr, nullptr, f);
}

long long lbve2d_time(const lbve2d_ctx *c) { return c ? c->t : -1; }
const char *lbve2d_last_error(const lbve2d_ctx *c) { return c ? c->err.c_str() : g_err2.c_str(); }

} // extern "C"

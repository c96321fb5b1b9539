// lbve_noalloc.cu -- time steps on caller-owned device buffers without any device
// allocation (lbve_step_noalloc in include/lbve.h).
//
// The split step needs one intermediate field besides the caller's state: the velocity
// u^t that the stream-collide kernel writes and the stress kernel reads.  Here it lives
// in a file-scope device array of fixed size instead of memory allocated per call, so
// that callers that may not allocate device memory can still advance a solve.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbve_host.h"
#include "lbve_launch.h"

using namespace lbve;

namespace {

// Largest grid (cells) the static scratch serves: 3 velocity components of up to 8 bytes.
constexpr long long kNoallocMaxCells = LBVE_NOALLOC_MAX_CELLS;

// The velocity scratch and the neighbour masks derived from the caller's flags.  Every
// GPU that loads the library holds them until exit.
static __device__ __align__(256) double g_noalloc_u[3 * kNoallocMaxCells];
static __device__ __align__(256) uint32_t g_noalloc_mask[kNoallocMaxCells];
// Zero-valued particle table: a particle flag in the caller's field then acts as a
// resting wall instead of dereferencing a missing table.
static __device__ __align__(256) PartDev g_noalloc_parts[MAX_PART];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void *g_u_addr[kMaxDevices] = {nullptr};
void *g_parts_addr[kMaxDevices] = {nullptr};
void *g_mask_addr[kMaxDevices] = {nullptr};
thread_local std::string g_err;

lbve_status fail(lbve_status s, const std::string &m) {
    g_err = m;
    return s;
}

const KernelTable *table_for(int prec) {
    switch (prec) {
    case LBVE_F64:
        return table_f64();
    case LBVE_F32:
        return table_f32();
    case LBVE_F16_SHIFTED:
        return table_f16();
    case LBVE_BF16_SHIFTED:
        return table_bf16();
    default:
        return nullptr;
    }
}

} // namespace

extern "C" {

lbve_status lbve_step_noalloc(const lbve_params *p, void *f, void *tau_a, void *tau_b, const uint8_t *flags,
                              const double *wall_vel, int n_wall, long long t0, int nsteps, void *cuda_stream) {
    std::string why;
    if (!params_valid(p, why)) return fail(LBVE_EINVAL, why);
    if (!f || !tau_a || !tau_b || !flags) return fail(LBVE_EINVAL, "a device buffer is NULL");
    if (nsteps < 0 || t0 < 0) return fail(LBVE_EINVAL, "nsteps and t0 must be >= 0");
    if (p->fene_L2 > 0.0) return fail(LBVE_EINVAL, "lbve_step_noalloc does not run FENE-P");
    if (p->schedule != LBVE_SCHED_AUTO && p->schedule != LBVE_SCHED_SPLIT)
        return fail(LBVE_EINVAL, "lbve_step_noalloc runs the split schedule only (schedule AUTO or SPLIT)");
    if (n_wall < 0 || n_wall > MAX_WALL || (n_wall > 0 && !wall_vel))
        return fail(LBVE_EINVAL, "n_wall must be in [0, 16] with wall_vel given");
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n > kNoallocMaxCells) return fail(LBVE_EINVAL, "grid exceeds LBVE_NOALLOC_MAX_CELLS cells");
    if (nsteps == 0) return LBVE_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBVE_EINVAL, "device index out of range");
    void *u_scratch, *parts, *mask;
    {
        // once per device, with that device current: the device address of the arrays
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_u_addr[dev]) {
            void *a = nullptr, *b = nullptr;
            e = cudaGetSymbolAddress(&a, g_noalloc_u);
            if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = cudaGetSymbolAddress(&b, g_noalloc_parts);
            if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            void *m = nullptr;
            e = cudaGetSymbolAddress(&m, g_noalloc_mask);
            if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_parts_addr[dev] = b;
            g_mask_addr[dev] = m;
            g_u_addr[dev] = a;
        }
        u_scratch = g_u_addr[dev];
        parts = g_parts_addr[dev];
        mask = g_mask_addr[dev];
    }
    DevState d;
    d.g.nx = p->nx;
    d.g.ny = p->ny;
    d.g.nz = p->nz;
    for (int k = 0; k < 3; ++k) d.g.per[k] = p->periodic[k] ? 1 : 0;
    d.g.n = n;
    d.g.np = (n + 63) / 64 * 64;
    fill_phys(*p, d.ph);
    for (int k = 0; k < MAX_WALL; ++k)
        for (int a = 0; a < 3; ++a) d.ph.wall_vel[k][a] = k < n_wall ? wall_vel[3 * k + a] : 0.0;
    d.f = f;
    d.tau[0] = tau_a;
    d.tau[1] = tau_b;
    d.u[0] = d.u[1] = u_scratch;  // fully written by the stream-collide kernel before the stress kernel reads it
    d.ucur = 0;
    d.mask = (uint32_t *)mask;     // rebuilt from the caller's flags below, before any step kernel
    d.flag = const_cast<uint8_t *>(flags);
    d.parts = (PartDev *)parts;
    d.cur = 0;
    d.block_x = default_block_x(*p);
    d.fv_zchunk = 0;
    d.step = (unsigned)t0;
    const KernelTable *kt = table_for(p->pdf_prec);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    e = kt->build_mask(d, 0, 0, 0, p->nx, p->ny, p->nz, s);
    if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("mask kernel: ") + cudaGetErrorString(e));
    for (int k = 0; k < nsteps; ++k) {
        const int parity = (int)((t0 + k) & 1);
        d.step = (unsigned)(t0 + k);
        e = kt->lb(d, parity, s);
        if (e == cudaSuccess) e = kt->fv(d, s);
        if (e != cudaSuccess) return fail(LBVE_ECUDA, std::string("step kernels: ") + cudaGetErrorString(e));
        d.cur ^= 1;
    }
    return LBVE_OK;
}

const char *lbve_noalloc_last_error(void) { return g_err.c_str(); }

} // extern "C"

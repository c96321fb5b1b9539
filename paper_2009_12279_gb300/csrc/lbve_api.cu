// lbve_api.cu -- host implementation of the C ABI declared in include/lbve.h.
//
// A context owns the device state of one solve (PDFs, stress ping-pong, velocity,
// flags, particles, boundary-link list) and enqueues the step kernels of the
// per-precision kernel tables on its stream.
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbve.h"
#include "lbve_host.h"
#include "lbve_launch.h"

using namespace lbve;

struct lbve_ctx {
    lbve_params p;
    cudaStream_t stream = nullptr;
    lbve_alloc_fn alloc = nullptr;
    lbve_free_fn dealloc = nullptr;
    void *user = nullptr;
    const KernelTable *kt = nullptr;
    DevState d;
    long long t = 0;
    std::string err;
    std::vector<std::pair<void *, size_t>> blocks;
    // boundary links into tracked bodies, one segment per body:
    // [wall-class links (host-built) | particle 0 capacity | particle 1 capacity | ...]
    std::vector<long long> wall_links;
    std::vector<int> wall_seg_begin, wall_seg_count, wall_seg_flag;
    long long *links = nullptr;  // device, capacity links_cap
    size_t links_cap = 0;
    double *contrib = nullptr;   // device, 8 doubles per entry (per link, or per partial)
    size_t contrib_cap = 0;      // entries
    int lb_tx = 0, fv_tx = 0;    // tile widths in a pool's batched kernels (0: default by nx)
    int *seg_begin = nullptr;    // device, kMaxBodies each
    int *seg_count = nullptr;
    int *seg_flag = nullptr;
    int nbody = 0, max_seg_len = 0;
    int *part_cap = nullptr;     // device, link capacity per particle
    std::vector<int> part_cap_host;
    uint8_t *pkind = nullptr, *pnf = nullptr;  // fill/drain scratch (largest particle box)
    double *pdelta = nullptr;
    int *pconv = nullptr;
    size_t pscratch_cells = 0;
    double *pdiag = nullptr;     // device: dropped stress (6), destroyed, created
    double *body_F = nullptr;    // device, 256 x 3 forces of the last step
    double *red = nullptr;       // device reduction scratch
    size_t red_cap = 0;
    double *red_out = nullptr;   // device, 6 doubles
    bool geometry_set = false;
    int nparts = 0;
    PartDev parts_host[MAX_PART];
    // kernel timing (event pairs recorded around launches while enabled)
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<int> ev_kind;  // kind of each recorded pair, in order
    size_t ev_used = 0;
    double kt_ms[LBVE_KT_COUNT] = {0};
    long long kt_count[LBVE_KT_COUNT] = {0};
    // steady-state residual
    void *usnap = nullptr;
    double *res_partial = nullptr;
    lbve_pool *pool = nullptr;
    // instability flag: mapped page-locked word set by the stream-collide (d.bad is its
    // device address); read by the host without synchronising
    unsigned *h_bad = nullptr;
    // z-slab stepping: AA parity of the last stream-collide, and a stream-collide whose
    // stress update (lbve_step_phase 1) is still to come
    int last_lb_parity = 0;
    bool phase_pending = false;
};

namespace {
// Process-wide record of tuned schedules: single solves by (precision, nx, ny, nz) ->
// (stream-collide block width, stress z-planes per block); pool tiles by (precision, nx)
// -> (stream-collide tile width, stress tile width).
std::mutex g_tune_mu;
std::map<std::array<int, 4>, std::array<int, 2>> g_tuned_ctx;
std::map<std::array<int, 2>, std::array<int, 2>> g_tuned_tiles;

bool tuned_ctx(const lbve_params &p, int &bx, int &zc) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_ctx.find({p.pdf_prec, p.nx, p.ny, p.nz});
    if (it == g_tuned_ctx.end()) return false;
    bx = it->second[0];
    zc = it->second[1];
    return true;
}
bool tuned_tiles(int prec, int nx, int &lb_tx, int &fv_tx) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_tiles.find({prec, nx});
    if (it == g_tuned_tiles.end()) return false;
    lb_tx = it->second[0];
    fv_tx = it->second[1];
    return true;
}
} // namespace

namespace {

std::string g_create_error;

const char *kStatusNames[] = {"LBVE_OK",        "LBVE_EINVAL",   "LBVE_ENOMEM", "LBVE_ECUDA",
                              "LBVE_EUNSTABLE", "LBVE_ETIMEOUT", "LBVE_ESTATE"};

lbve_status fail(lbve_ctx *c, lbve_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

// The instability flag of a context (set by a stream-collide of an earlier call; the
// host sees it once that kernel has written it, without synchronising).
bool unstable(const lbve_ctx *c) { return c->h_bad && *(volatile const unsigned *)c->h_bad != 0u; }
// The flag value 2: a bounded wait of the row-pipelined stream-collide gave up.
bool timed_out(const lbve_ctx *c) { return c->h_bad && *(volatile const unsigned *)c->h_bad == 2u; }
lbve_status flag_status(const lbve_ctx *c) { return timed_out(c) ? LBVE_ETIMEOUT : LBVE_EUNSTABLE; }
std::string unstable_message(const lbve_ctx *c) {
    if (timed_out(c))
        return "a stream-collide block gave up waiting for its shared-memory copies at or before step " +
               std::to_string(c->t);
    return "instability detected at or before step " + std::to_string(c->t) +
           ": a fluid cell had rho <= 0, |u|^2 >= 1/3 or a NaN";
}
void clear_unstable(lbve_ctx *c) {
    if (c->h_bad) *(volatile unsigned *)c->h_bad = 0u;
}

lbve_status cuda_fail(lbve_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (c) c->err = m;
    return e == cudaErrorMemoryAllocation ? LBVE_ENOMEM : LBVE_ECUDA;
}

#define CK(call, where)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

long long padded(long long n) { return (n + 63) / 64 * 64; }

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

size_t pdf_bytes_of(int prec) { return prec == LBVE_F64 ? 8 : (prec == LBVE_F32 ? 4 : 2); }
size_t real_bytes_of(int prec) { return prec == LBVE_F64 ? 8 : 4; }

bool valid_params(const lbve_params *p, std::string &why) {
    if (!p) return why = "params is NULL", false;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return why = "grid dimensions must be >= 1", false;
    if (p->ny > 65535 || p->nz > 65535) return why = "ny and nz must be <= 65535", false;
    if ((long long)p->nx * p->ny * p->nz > 2147483647LL) return why = "grids are limited to 2^31 - 1 cells", false;
    if (!(p->eta > 0.0)) return why = "eta must be > 0", false;
    if (!(p->beta >= 0.0 && p->beta < 1.0)) return why = "beta must be in [0, 1)", false;
    if (!(p->rho0 > 0.0)) return why = "rho0 must be > 0", false;
    if (p->beta > 0.0 && !(p->lambda_p > 0.0)) return why = "lambda_p must be > 0 when beta > 0", false;
    if (p->pdf_prec < LBVE_F64 || p->pdf_prec > LBVE_BF16_SHIFTED) return why = "unknown pdf_prec", false;
    if (p->pdf_scale_log2 < -1 || p->pdf_scale_log2 > 24) return why = "pdf_scale_log2 out of range", false;
    if (p->fv_terms < 0 || p->fv_terms > 15) return why = "fv_terms out of range", false;
    if (!(p->giesekus_alpha >= 0.0 && p->giesekus_alpha <= 0.5)) return why = "giesekus_alpha must be in [0, 1/2]", false;
    if (!(p->fene_L2 == 0.0 || p->fene_L2 > 3.0)) return why = "fene_L2 must be 0 (Oldroyd-B) or > 3", false;
    if (p->fene_L2 > 0.0 && !(p->beta > 0.0)) return why = "FENE-P needs a polymer (beta > 0)", false;
    if (p->fene_L2 > 0.0 && p->giesekus_alpha != 0.0) return why = "FENE-P and Giesekus cannot be combined", false;
    if (p->schedule < LBVE_SCHED_AUTO || p->schedule > LBVE_SCHED_PIPELINED) return why = "unknown schedule", false;
    if (p->fene_L2 > 0.0 && p->schedule == LBVE_SCHED_FUSED)
        return why = "FENE-P runs on the split schedule only", false;
    if (p->block_x != 0 && p->block_x != 32 && p->block_x != 64 && p->block_x != 128)
        return why = "block_x must be 0, 32, 64 or 128", false;
    if (!(p->magic >= 0.0)) return why = "magic must be >= 0", false;
    const double eta_n = (1.0 - p->beta) * p->eta;
    if (!(eta_n / p->rho0 > 0.0)) return why = "Newtonian viscosity must be > 0", false;
    return true;
}

void *dev_alloc(lbve_ctx *c, size_t bytes) {
    void *ptr = nullptr;
    if (c->alloc) {
        ptr = c->alloc(bytes, (void *)c->stream, c->user);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) c->blocks.push_back({ptr, bytes});
    return ptr;
}

void dev_free(lbve_ctx *c, void *ptr) {
    if (!ptr) return;
    for (size_t k = 0; k < c->blocks.size(); ++k) {
        if (c->blocks[k].first == ptr) {
            if (c->dealloc)
                c->dealloc(ptr, c->blocks[k].second, (void *)c->stream, c->user);
            else
                cudaFree(ptr);
            c->blocks.erase(c->blocks.begin() + (long)k);
            return;
        }
    }
}

void set_phys(lbve_ctx *c) { lbve::fill_phys(c->p, c->d.ph); }

} // namespace

void lbve::fill_phys(const lbve_params &p, Phys<double> &ph) {
    std::memset(&ph, 0, sizeof(ph));
    // TRT rates from the viscosity (Sec. "Lattice Boltzmann"): rates, magic product.
    const double eta_n = (1.0 - p.beta) * p.eta;
    const double nu_n = eta_n / p.rho0;
    const double magic = p.magic > 0.0 ? p.magic : 3.0 / 16.0;
    ph.omega_p = 1.0 / (3.0 * nu_n + 0.5);
    const double tp = 1.0 / ph.omega_p - 0.5;
    ph.omega_m = 1.0 / (magic / tp + 0.5);
    ph.A = 3.0 * (1.0 - 0.5 * ph.omega_m);
    ph.B = 1.0 - 0.5 * ph.omega_p;
    const double eta_p = p.beta * p.eta;
    ph.ep_l = p.beta > 0.0 ? eta_p / p.lambda_p : 0.0;
    ph.inv_l = p.lambda_p > 0.0 ? 1.0 / p.lambda_p : 0.0;
    for (int k = 0; k < 3; ++k) ph.g[k] = p.body_force[k];
    ph.rho0 = p.pdf_prec == LBVE_F64 ? 0.0 : p.rho0;
    ph.rho_ref = p.rho0;
    // the storage scale only serves FP16 (5-bit exponent); FP32 and BF16 store unscaled
    int k = p.pdf_scale_log2 < 0 ? 15 : p.pdf_scale_log2;
    if (p.pdf_prec != LBVE_F16_SHIFTED) k = 0;
    ph.scale = std::ldexp(1.0, k);
    ph.inv_scale = std::ldexp(1.0, -k);
    const int base = LBVE_FV_FLUX | LBVE_FV_SOURCE;
    const int terms = (p.fv_terms & base) == 0 ? (p.fv_terms | base) : p.fv_terms;
    ph.flux_on = (terms & LBVE_FV_FLUX) != 0;
    ph.src_on = (terms & LBVE_FV_SOURCE) != 0;
    ph.ctu_on = (terms & LBVE_FV_CTU) != 0;
    ph.divu_on = (terms & LBVE_FV_DIVU) != 0;
    ph.gk = p.beta > 0.0 ? p.giesekus_alpha / (p.beta * p.eta) : 0.0;
    ph.fene = p.fene_L2 > 0.0 ? 1 : 0;
    ph.fene_L2 = p.fene_L2;
    ph.eta_p = eta_p;
    ph.lam = p.lambda_p;
}

bool lbve::params_valid(const lbve_params *p, std::string &why) { return valid_params(p, why); }

int lbve::default_block_x(const lbve_params &p) {
    int bx = p.block_x > 0 ? p.block_x : 64;  // 64 x 2 measured ~1 % ahead of 32 x 4 at 512^3
    if (bx > 128) bx = 128;
    while (bx > 32 && bx / 2 >= p.nx) bx /= 2;
    return bx;
}

namespace {

// ---------------------------------------------------------------------------------
// small kernels that do not depend on the storage type
// ---------------------------------------------------------------------------------

// Sum the momentum-exchange contributions of each body segment in link order (FP64
// parity mode, launched with one thread per body: the sequential order of a plain loop;
// with more threads a fixed-shape block reduction).
__global__ void k_body_reduce(const double *__restrict__ contrib, const int *__restrict__ seg_begin,
                              const int *__restrict__ seg_count, const int *__restrict__ seg_flag, int nbody,
                              double *__restrict__ body_F, PartDev *__restrict__ parts) {
    const int b = blockIdx.x;
    if (b >= nbody) return;
    const int beg = seg_begin[b], end = seg_begin[b] + seg_count[b];
    __shared__ double sh[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int T = blockDim.x;
    // thread t sums links beg + t, beg + t + T, ... (coalesced; one thread: link order)
    for (int l = beg + (int)threadIdx.x; l < end; l += T)
        for (int k = 0; k < 6; ++k) acc[k] += contrib[(long long)l * 8 + k];
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int fl = seg_flag[b];
        for (int k = 0; k < 3; ++k) body_F[fl * 3 + k] = sh[k][0];
        if (fl >= FLAG_PART0 && fl < FLAG_PART0 + MAX_PART) {
            PartDev &P = parts[fl - FLAG_PART0];
            for (int k = 0; k < 3; ++k) {
                P.Fme[k] = sh[k][0];
                P.Tme[k] = sh[3 + k][0];
            }
        }
    }
}

// Per-body sums of the reduced modes' momentum-exchange partials (gx per body, first
// ceil(count / 128) used): warp w sums component w over partials lane, lane + 32, ...,
// then a fixed shuffle tree.  Deterministic.
__global__ void __launch_bounds__(192) k_body_partials(const double *__restrict__ part, int gx,
                                                       const int *__restrict__ seg_count,
                                                       const int *__restrict__ seg_flag, int nbody,
                                                       double *__restrict__ body_F, PartDev *__restrict__ parts) {
    const int b = blockIdx.x;
    if (b >= nbody) return;
    const int n = (seg_count[b] + 127) / 128;
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc += part[((long long)b * gx + j) * 8 + w];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    __shared__ double tot[6];
    if (lane == 0) tot[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int fl = seg_flag[b];
        for (int k = 0; k < 3; ++k) body_F[fl * 3 + k] = tot[k];
        if (fl >= FLAG_PART0 && fl < FLAG_PART0 + MAX_PART) {
            PartDev &P = parts[fl - FLAG_PART0];
            for (int k = 0; k < 3; ++k) {
                P.Fme[k] = tot[k];
                P.Tme[k] = tot[3 + k];
            }
        }
    }
}

// Device address of a host buffer that is page-locked and mapped (cudaHostAlloc or
// cudaHostRegister under unified addressing), else nullptr (pageable memory is staged).
void *mapped_host(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Fault in the pages of a pageable host output buffer before a device-to-host copy into
// it: one write per page.  Copies into pages that were never touched (fresh calloc/mmap
// memory) ran 10-15x slower than into touched ones, the pages being brought in one by one
// on the copy path.  The buffer is output-only, so the bytes written here are overwritten.
void prefault_output(void *p, size_t bytes) {
    if (!p || bytes == 0) return;
    // plain pageable host memory only (not device, managed or page-locked memory)
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (at.type != cudaMemoryTypeUnregistered) return;
    static const size_t page = [] {
        const long v = sysconf(_SC_PAGESIZE);
        return v > 0 ? (size_t)v : (size_t)4096;
    }();
    volatile unsigned char *b = (volatile unsigned char *)p;
    for (size_t o = 0; o < bytes; o += page) b[o] = 0;
    b[bytes - 1] = 0;
}

// Advance a pool's device step counter (after each step's stream-collide).
__global__ void k_step_count(unsigned *dstep) { *dstep += 1u; }

// Launch the per-body force / torque sums of a context's momentum exchange.
cudaError_t body_sums(const lbve_ctx *c, PartDev *parts, cudaStream_t st) {
    if (c->p.pdf_prec == LBVE_F64)
        k_body_reduce<<<c->nbody, 1, 0, st>>>(c->contrib, c->seg_begin, c->seg_count, c->seg_flag, c->nbody,
                                              c->body_F, parts);
    else
        k_body_partials<<<c->nbody, 192, 0, st>>>(c->contrib, (c->max_seg_len + 127) / 128, c->seg_count,
                                                  c->seg_flag, c->nbody, c->body_F, parts);
    return cudaGetLastError();
}

__global__ void k_final_sum(const double *__restrict__ partial, long long nblocks, double *__restrict__ out) {
    __shared__ double sh[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 6; ++k) acc[k] = k == 5 ? fmax(acc[k], partial[b * 6 + k]) : acc[k] + partial[b * 6 + k];
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 6; ++k)
                sh[k][threadIdx.x] = k == 5 ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + s])
                                            : sh[k][threadIdx.x] + sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Host-side list of links (fluid cell r, direction i with r + c_i a wall-class cell),
// ordered by flag value, then cell, then direction (the order of a plain cell loop
// within each body).  Built from the wall-class cells, so its cost is O(wall cells).
void build_wall_links(lbve_ctx *c, const uint8_t *fl, bool any_wall) {
    std::vector<long long> &links = c->wall_links;
    std::vector<int> &seg = c->wall_seg_begin, &seg_flag = c->wall_seg_flag, &seg_count = c->wall_seg_count;
    links.clear();
    seg.clear();
    seg_flag.clear();
    seg_count.clear();
    if (!any_wall) return;
    static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const long long n = (long long)nx * ny * nz;
    std::vector<std::pair<int, long long>> tmp;  // (flag, (r << 5) | i)
    for (long long rw = 0; rw < n; ++rw) {
        const uint8_t f = fl[rw];
        if (f < FLAG_WALL0 || f >= FLAG_WALL0 + MAX_WALL) continue;
        const int x = (int)(rw % nx), y = (int)((rw / nx) % ny), z = (int)(rw / ((long long)nx * ny));
        for (int i = 1; i < Q; ++i) {
            // fluid cell r with r + c_i = rw
            int xq = x - CX[i], yq = y - CY[i], zq = z - CZ[i];
            if (xq < 0 || xq >= nx || yq < 0 || yq >= ny || zq < 0 || zq >= nz) {
                if (!c->p.periodic[0] && (xq < 0 || xq >= nx)) continue;
                if (!c->p.periodic[1] && (yq < 0 || yq >= ny)) continue;
                if (!c->p.periodic[2] && (zq < 0 || zq >= nz)) continue;
                xq = (xq + nx) % nx;
                yq = (yq + ny) % ny;
                zq = (zq + nz) % nz;
            }
            const long long r = xq + (long long)nx * (yq + (long long)ny * zq);
            if (c->d.zhi > 0 && (zq < c->d.zlo || zq >= c->d.zhi)) continue;  // a ghost plane of a z-slab
            if (fl[r] == FLAG_FLUID) tmp.push_back({(int)f, (r << 5) | i});
        }
    }
    std::sort(tmp.begin(), tmp.end());
    for (size_t k = 0; k < tmp.size(); ++k) {
        if (k == 0 || tmp[k].first != tmp[k - 1].first) {
            seg.push_back((int)links.size());
            seg_flag.push_back(tmp[k].first);
            seg_count.push_back(0);
        }
        links.push_back(tmp[k].second);
        seg_count.back()++;
    }
}

constexpr int kMaxBodies = 128;

// Lay out the link array (wall links, then one fixed-capacity segment per particle),
// upload the wall links and the segment tables, and build the particles' links.
lbve_status layout_links(lbve_ctx *c) {
    size_t total = c->wall_links.size();
    for (int cap : c->part_cap_host) total += (size_t)cap;
    if (total > c->links_cap) {
        dev_free(c, c->links);
        dev_free(c, c->contrib);
        c->links = nullptr;
        c->contrib = nullptr;
        const size_t cap = std::max<size_t>(total, 1024);
        c->links = (long long *)dev_alloc(c, cap * sizeof(long long));
        c->contrib = (double *)dev_alloc(c, cap * 8 * sizeof(double));
        if (!c->links || !c->contrib) return fail(c, LBVE_ENOMEM, "link list allocation failed");
        c->links_cap = cap;
        c->contrib_cap = cap;
    }
    if (!c->wall_links.empty())
        CK(cudaMemcpyAsync(c->links, c->wall_links.data(), c->wall_links.size() * sizeof(long long),
                           cudaMemcpyHostToDevice, c->stream),
           "upload links");
    std::vector<int> beg(c->wall_seg_begin), cnt(c->wall_seg_count), flg(c->wall_seg_flag);
    int off = (int)c->wall_links.size();
    int mx = 0;
    for (int v : cnt) mx = std::max(mx, v);
    for (int p = 0; p < c->nparts; ++p) {
        beg.push_back(off);
        cnt.push_back(0);
        flg.push_back(FLAG_PART0 + p);
        off += c->part_cap_host[p];
        mx = std::max(mx, c->part_cap_host[p]);
    }
    c->nbody = (int)beg.size();
    c->max_seg_len = mx;
    if (c->nbody > kMaxBodies) return fail(c, LBVE_EINVAL, "too many tracked bodies");
    // the reduced modes keep one partial per (body, block of 128 links) in contrib
    const size_t parts_needed = (size_t)c->nbody * (size_t)((mx + 127) / 128);
    if (parts_needed > c->contrib_cap) {
        dev_free(c, c->contrib);
        c->contrib = (double *)dev_alloc(c, parts_needed * 8 * sizeof(double));
        if (!c->contrib) return fail(c, LBVE_ENOMEM, "momentum-exchange partials allocation failed");
        c->contrib_cap = parts_needed;
    }
    if (c->nbody > 0) {
        CK(cudaMemcpyAsync(c->seg_begin, beg.data(), beg.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "seg");
        CK(cudaMemcpyAsync(c->seg_count, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "seg");
        CK(cudaMemcpyAsync(c->seg_flag, flg.data(), flg.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "seg");
    }
    if (c->nparts > 0) {
        CK(cudaMemcpyAsync(c->part_cap, c->part_cap_host.data(), sizeof(int) * c->nparts, cudaMemcpyHostToDevice,
                           c->stream),
           "part cap");
        CK(c->kt->particle_links(c->d, c->nparts, c->links, c->seg_begin, c->seg_count, (int)c->wall_seg_begin.size(),
                                 c->part_cap, c->stream),
           "particle links");
    }
    CK(cudaStreamSynchronize(c->stream), "links sync");
    return LBVE_OK;
}

lbve_status create_impl(const lbve_params *p, void *stream, lbve_alloc_fn alloc, lbve_free_fn dealloc, void *user,
                        lbve_ctx **out) {
    if (!out) return LBVE_EINVAL;
    *out = nullptr;
    std::string why;
    if (!valid_params(p, why)) {
        g_create_error = why;
        return LBVE_EINVAL;
    }
    lbve_ctx *c = new (std::nothrow) lbve_ctx();
    if (!c) return LBVE_ENOMEM;
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    c->alloc = alloc;
    c->dealloc = dealloc;
    c->user = user;
    c->kt = table_for(p->pdf_prec);
    std::memset(&c->d, 0, sizeof(c->d));
    Geo &g = c->d.g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    for (int k = 0; k < 3; ++k) g.per[k] = p->periodic[k] ? 1 : 0;
    g.n = (long long)p->nx * p->ny * p->nz;
    g.np = padded(g.n);
    c->d.block_x = lbve::default_block_x(*p);
    c->d.auto_kernels = p->schedule == LBVE_SCHED_AUTO ? 1 : (p->schedule == LBVE_SCHED_PIPELINED ? 2 : 0);
    if (p->block_x == 0) {  // a schedule tuned for this shape earlier in the process
        int bx = 0, zc = 0;
        if (tuned_ctx(*p, bx, zc)) {
            c->d.block_x = bx;
            c->d.fv_zchunk = zc;
        }
    }
    set_phys(c);
    const long long np = g.np;
    c->d.f = dev_alloc(c, (size_t)Q * np * c->kt->pdf_bytes);
    c->d.tau[0] = dev_alloc(c, (size_t)6 * np * c->kt->real_bytes);
    c->d.tau[1] = dev_alloc(c, (size_t)6 * np * c->kt->real_bytes);
    c->d.u[0] = dev_alloc(c, (size_t)3 * np * c->kt->real_bytes);
    c->d.u[1] = dev_alloc(c, (size_t)3 * np * c->kt->real_bytes);
    c->d.ucur = 0;
    c->d.mask = (uint32_t *)dev_alloc(c, (size_t)np * sizeof(uint32_t));
    c->d.flag = (uint8_t *)dev_alloc(c, (size_t)np);
    c->d.parts = (PartDev *)dev_alloc(c, sizeof(PartDev) * MAX_PART);
    c->seg_begin = (int *)dev_alloc(c, sizeof(int) * kMaxBodies);
    c->seg_count = (int *)dev_alloc(c, sizeof(int) * kMaxBodies);
    c->seg_flag = (int *)dev_alloc(c, sizeof(int) * kMaxBodies);
    c->part_cap = (int *)dev_alloc(c, sizeof(int) * MAX_PART);
    c->pdiag = (double *)dev_alloc(c, sizeof(double) * 8);
    c->body_F = (double *)dev_alloc(c, sizeof(double) * 256 * 3);
    c->red_out = (double *)dev_alloc(c, sizeof(double) * 8);
    if (!c->d.f || !c->d.tau[0] || !c->d.tau[1] || !c->d.u[0] || !c->d.u[1] || !c->d.mask || !c->d.flag || !c->d.parts || !c->seg_begin || !c->seg_count ||
        !c->seg_flag || !c->part_cap || !c->pdiag ||
        !c->body_F || !c->red_out) {
        g_create_error = "device allocation failed";
        lbve_destroy(c);
        return LBVE_ENOMEM;
    }
    cudaError_t e = cudaHostAlloc((void **)&c->h_bad, sizeof(unsigned), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *c->h_bad = 0u;
        void *dbad = nullptr;
        e = cudaHostGetDevicePointer(&dbad, c->h_bad, 0);
        c->d.bad = (unsigned *)dbad;
    } else {
        c->h_bad = nullptr;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d.flag, 0, (size_t)np, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d.u[0], 0, (size_t)3 * np * c->kt->real_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d.u[1], 0, (size_t)3 * np * c->kt->real_bytes, c->stream);
    if (e == cudaSuccess) e = c->kt->build_mask(c->d, 0, 0, 0, g.nx, g.ny, g.nz, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d.tau[1], 0, (size_t)6 * np * c->kt->real_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d.parts, 0, sizeof(PartDev) * MAX_PART, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->body_F, 0, sizeof(double) * 256 * 3, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->pdiag, 0, sizeof(double) * 8, c->stream);
    if (e == cudaSuccess) e = c->kt->init(c->d, nullptr, nullptr, nullptr, 0, g.n, g.n, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("initialisation failed: ") + cudaGetErrorString(e);
        lbve_destroy(c);
        return LBVE_ECUDA;
    }
    *out = c;
    return LBVE_OK;
}

// Start / stop a timed launch of the given kind (no-ops while timing is off).
cudaError_t timed_begin(lbve_ctx *c, int kind) {
    if (!c->timing) return cudaSuccess;
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t a, b;
        cudaError_t e = cudaEventCreate(&a);
        if (e != cudaSuccess) return e;
        e = cudaEventCreate(&b);
        if (e != cudaSuccess) return e;
        c->ev_pool.push_back({a, b});
    }
    if (c->ev_kind.size() <= c->ev_used) c->ev_kind.resize(c->ev_used + 1);
    c->ev_kind[c->ev_used] = kind;
    return cudaEventRecord(c->ev_pool[c->ev_used].first, c->stream);
}

cudaError_t timed_end(lbve_ctx *c) {
    if (!c->timing) return cudaSuccess;
    cudaError_t e = cudaEventRecord(c->ev_pool[c->ev_used].second, c->stream);
    c->ev_used++;
    return e;
}

// Fold the recorded event pairs into the per-kind totals and recycle them.
cudaError_t harvest_times(lbve_ctx *c) {
    if (c->ev_used == 0) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    for (size_t k = 0; k < c->ev_used; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->ev_pool[k].first, c->ev_pool[k].second);
        if (e != cudaSuccess) return e;
        c->kt_ms[c->ev_kind[k]] += ms;
        c->kt_count[c->ev_kind[k]] += 1;
    }
    c->ev_used = 0;
    return cudaSuccess;
}

// Host <-> device transfers of the FP64 fields go through a bounded staging buffer in
// slabs of whole z-planes (10 doubles per cell: rho, u, tau).
constexpr size_t kStagingBytes = size_t(256) << 20;

int slab_planes(const lbve_ctx *c) {
    const long long plane = (long long)c->p.nx * c->p.ny;
    long long k = (long long)(kStagingBytes / (sizeof(double) * 10 * (size_t)plane));
    if (k < 1) k = 1;
    if (k > c->p.nz) k = c->p.nz;
    return (int)k;
}

} // namespace

extern "C" {

void lbve_default_params(lbve_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 16;
    p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
    p->eta = 1.0 / 6.0;
    p->beta = 0.5;
    p->lambda_p = 1000.0;
    p->rho0 = 1.0;
    p->magic = 3.0 / 16.0;
    p->pdf_prec = LBVE_F32;
    p->pdf_scale_log2 = -1;
    p->fv_terms = LBVE_FV_FLUX | LBVE_FV_SOURCE;
    p->schedule = LBVE_SCHED_AUTO;
    p->block_x = 0;
}

size_t lbve_device_bytes(const lbve_params *p) {
    std::string why;
    if (!valid_params(p, why)) return 0;
    const long long np = padded((long long)p->nx * p->ny * p->nz);
    const size_t pb = pdf_bytes_of(p->pdf_prec), rb = real_bytes_of(p->pdf_prec);
    return (size_t)np * (Q * pb + 18 * rb + 1 + 4) + sizeof(PartDev) * MAX_PART + 32768;
}

lbve_status lbve_create(const lbve_params *p, void *cuda_stream, lbve_ctx **out) {
    return create_impl(p, cuda_stream, nullptr, nullptr, nullptr, out);
}

lbve_status lbve_create_with_allocator(const lbve_params *p, void *cuda_stream, lbve_alloc_fn alloc,
                                       lbve_free_fn dealloc, void *user, lbve_ctx **out) {
    if (!alloc || !dealloc) {
        g_create_error = "allocator callbacks must both be set";
        return LBVE_EINVAL;
    }
    return create_impl(p, cuda_stream, alloc, dealloc, user, out);
}

lbve_status lbve_destroy(lbve_ctx *c) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) lbve_pool_remove(c->pool, c);
    cudaStreamSynchronize(c->stream);
    for (auto &ev : c->ev_pool) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    while (!c->blocks.empty()) dev_free(c, c->blocks.back().first);
    if (c->h_bad) cudaFreeHost(c->h_bad);
    delete c;
    return LBVE_OK;
}

lbve_status lbve_set_geometry(lbve_ctx *c, const uint8_t *flags, const double *wall_vel, int n_wall) {
    if (!c) return LBVE_EINVAL;
    if (!flags) return fail(c, LBVE_EINVAL, "flags is NULL");
    if (c->nparts > 0) return fail(c, LBVE_ESTATE, "geometry must be set before particles are added");
    if (c->pool) return fail(c, LBVE_ESTATE, "geometry cannot change while the solve is in a pool");
    if (n_wall < 0 || n_wall > MAX_WALL || (n_wall > 0 && !wall_vel))
        return fail(c, LBVE_EINVAL, "n_wall must be in [0, 16] with wall_vel given");
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    // valid flags form the range [0, FLAG_WALL0 + n_wall): one (vectorisable) maximum
    // checks them all and tells whether any wall class is present
    uint8_t fmax = 0;
    for (long long r = 0; r < c->d.g.n; ++r) fmax = flags[r] > fmax ? flags[r] : fmax;
    if (fmax >= FLAG_WALL0 + n_wall) {
        for (long long r = 0; r < c->d.g.n; ++r) {
            if (flags[r] < FLAG_WALL0 + n_wall) continue;
            char b[128];
            std::snprintf(b, sizeof b, "flag %d at cell %lld is not fluid, no-slip or a declared wall class",
                          (int)flags[r], r);
            return fail(c, LBVE_EINVAL, b);
        }
    }
    // a non-periodic direction needs non-fluid first and last layers
    const int nn[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (c->p.periodic[a]) continue;
        if (a == 2 && c->d.zhi > 0) continue;  // a z-slab's outer planes are its ghost planes
        for (int side = 0; side < 2; ++side) {
            const int q = side ? nn[a] - 1 : 0;
            const int b1 = a == 0 ? ny : nx, b2 = a == 2 ? ny : nz;
            for (int j = 0; j < b2; ++j)
                for (int i = 0; i < b1; ++i) {
                    const int x = a == 0 ? q : i, y = a == 1 ? q : (a == 0 ? i : j), z = a == 2 ? q : j;
                    if (flags[x + (long long)nx * (y + (long long)ny * z)] == FLAG_FLUID)
                        return fail(c, LBVE_EINVAL, "fluid cell in the outer layer of a non-periodic direction");
                }
        }
    }
    for (int k = 0; k < MAX_WALL; ++k)
        for (int a = 0; a < 3; ++a) c->d.ph.wall_vel[k][a] = k < n_wall ? wall_vel[3 * k + a] : 0.0;
    CK(cudaMemcpyAsync(c->d.flag, flags, (size_t)c->d.g.n, cudaMemcpyHostToDevice, c->stream), "upload flags");
    CK(c->kt->build_mask(c->d, 0, 0, 0, c->p.nx, c->p.ny, c->p.nz, c->stream), "neighbour masks");
    build_wall_links(c, flags, fmax >= FLAG_WALL0);
    lbve_status s = layout_links(c);
    if (s != LBVE_OK) return s;
    // the caller's buffer may be pinned: the copy has to be done when the call returns
    CK(cudaStreamSynchronize(c->stream), "geometry sync");
    c->geometry_set = true;
    return LBVE_OK;
}

lbve_status lbve_init_fields(lbve_ctx *c, const double *rho, const double *u, const double *tau) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) return fail(c, LBVE_ESTATE, "fields cannot be reset while the solve is in a pool");
    const long long n = c->d.g.n, plane = (long long)c->p.nx * c->p.ny;
    {
        // page-locked buffers the device can address: one kernel reads them in place
        const double *drho = rho ? (const double *)mapped_host(rho) : nullptr;
        const double *du = u ? (const double *)mapped_host(u) : nullptr;
        const double *dtau = tau ? (const double *)mapped_host(tau) : nullptr;
        if ((!rho || drho) && (!u || du) && (!tau || dtau)) {
            c->d.cur = 0;
            CK(c->kt->init(c->d, drho, du, dtau, 0, n, n, c->stream), "init kernel");
            CK(cudaStreamSynchronize(c->stream), "init sync");
            clear_unstable(c);
            c->t = 0;
            return LBVE_OK;
        }
    }
    const int zs = slab_planes(c);
    const long long cap = plane * zs;
    double *st = (double *)dev_alloc(c, sizeof(double) * 10 * (size_t)cap);
    if (!st) return fail(c, LBVE_ENOMEM, "staging allocation failed");
    c->d.cur = 0;
    for (int z0 = 0; z0 < c->p.nz; z0 += zs) {
        const int z1 = std::min(c->p.nz, z0 + zs);
        const long long r0 = (long long)z0 * plane, cnt = (long long)(z1 - z0) * plane;
        double *srho = st, *su = st + cnt, *stau = st + 4 * cnt;
        if (rho) CK(cudaMemcpyAsync(srho, rho + r0, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream), "init copy");
        for (int k = 0; u && k < 3; ++k)
            CK(cudaMemcpyAsync(su + k * cnt, u + k * n + r0, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream),
               "init copy");
        for (int k = 0; tau && k < 6; ++k)
            CK(cudaMemcpyAsync(stau + k * cnt, tau + k * n + r0, sizeof(double) * cnt, cudaMemcpyHostToDevice,
                               c->stream),
               "init copy");
        CK(c->kt->init(c->d, rho ? srho : nullptr, u ? su : nullptr, tau ? stau : nullptr, r0, cnt, cnt, c->stream),
           "init kernel");
    }
    CK(cudaStreamSynchronize(c->stream), "init sync");
    dev_free(c, st);
    clear_unstable(c);
    c->t = 0;
    return LBVE_OK;
}

lbve_status lbve_init_fields_device(lbve_ctx *c, const double *rho, const double *u, const double *tau) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) return fail(c, LBVE_ESTATE, "fields cannot be reset while the solve is in a pool");
    c->d.cur = 0;
    CK(c->kt->init(c->d, rho, u, tau, 0, c->d.g.n, c->d.g.n, c->stream), "init kernel");
    // the instability flag restarts with the new fields, in stream order
    if (c->d.bad) CK(cudaMemsetAsync(c->d.bad, 0, sizeof(unsigned), c->stream), "flag reset");
    c->t = 0;
    return LBVE_OK;
}

lbve_status lbve_probe(lbve_ctx *c, const int64_t *cells, int count, double *out) {
    if (!c) return LBVE_EINVAL;
    if (count < 0 || (count > 0 && (!cells || !out))) return fail(c, LBVE_EINVAL, "bad probe arguments");
    if (count == 0) return LBVE_OK;
    for (int k = 0; k < count; ++k)
        if (cells[k] < 0 || cells[k] >= c->d.g.n) return fail(c, LBVE_EINVAL, "probe cell index out of range");
    void *dc = dev_alloc(c, sizeof(long long) * (size_t)count);
    double *dout = (double *)dev_alloc(c, sizeof(double) * 29 * (size_t)count);
    if (!dc || !dout) {
        dev_free(c, dc);
        dev_free(c, dout);
        return fail(c, LBVE_ENOMEM, "probe staging allocation failed");
    }
    CK(cudaMemcpyAsync(dc, cells, sizeof(long long) * (size_t)count, cudaMemcpyHostToDevice, c->stream), "probe copy");
    CK(c->kt->probe(c->d, (int)(c->t & 1), (const long long *)dc, count, dout, c->stream), "probe kernel");
    CK(cudaMemcpyAsync(out, dout, sizeof(double) * 29 * (size_t)count, cudaMemcpyDeviceToHost, c->stream), "probe out");
    CK(cudaStreamSynchronize(c->stream), "probe sync");
    dev_free(c, dc);
    dev_free(c, dout);
    return LBVE_OK;
}

lbve_status lbve_add_particle(lbve_ctx *c, const double X[3], double R, double rho_p, const double v[3],
                              const double w[3], const double Fext[3], const double Text[3], int *id) {
    if (!c) return LBVE_EINVAL;
    if (!X) return fail(c, LBVE_EINVAL, "X is NULL");
    if (!(R > 0.0) || !(rho_p > 0.0)) return fail(c, LBVE_EINVAL, "radius and density must be > 0");
    if (c->nparts >= MAX_PART) return fail(c, LBVE_ESTATE, "too many particles");
    if (c->pool) return fail(c, LBVE_ESTATE, "particles cannot be added while the solve is in a pool");
    if (c->p.fene_L2 > 0.0) return fail(c, LBVE_ESTATE, "moving particles are not combined with FENE-P");
    if (c->d.zhi > 0) return fail(c, LBVE_ESTATE, "moving particles are not combined with a z-slab");
    const int nn[3] = {c->p.nx, c->p.ny, c->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(X[a])) return fail(c, LBVE_EINVAL, "X must be finite");
        if (2.0 * R + 6.0 > nn[a]) return fail(c, LBVE_EINVAL, "particle too large for the domain");
    }
    PartDev P;
    std::memset(&P, 0, sizeof(P));
    for (int a = 0; a < 3; ++a) {
        P.X[a] = X[a];
        P.v[a] = v ? v[a] : 0.0;
        P.w[a] = w ? w[a] : 0.0;
        P.Fext[a] = Fext ? Fext[a] : 0.0;
        P.Text[a] = Text ? Text[a] : 0.0;
    }
    P.R = R;
    P.rho_p = rho_p;
    P.m = rho_p * (4.0 / 3.0) * M_PI * R * R * R;
    P.I = 0.4 * P.m * R * R;
    P.changed = 1;
    const int p = c->nparts;
    // scratch for fill/drain (box with margin 3) and the link capacity (box with margin 2)
    const long long side3 = particle_box_side(R, 3), side2 = particle_box_side(R, 2);
    const size_t cells3 = (size_t)(side3 * side3 * side3);
    if (cells3 > c->pscratch_cells) {
        dev_free(c, c->pkind);
        dev_free(c, c->pnf);
        dev_free(c, c->pdelta);
        dev_free(c, c->pconv);
        c->pkind = (uint8_t *)dev_alloc(c, cells3);
        c->pnf = (uint8_t *)dev_alloc(c, cells3);
        c->pdelta = (double *)dev_alloc(c, sizeof(double) * 6 * cells3);
        c->pconv = (int *)dev_alloc(c, sizeof(int) * cells3);
        if (!c->pkind || !c->pnf || !c->pdelta || !c->pconv)
            return fail(c, LBVE_ENOMEM, "particle scratch allocation failed");
        CK(cudaMemsetAsync(c->pnf, 0, cells3, c->stream), "scratch clear");
        c->pscratch_cells = cells3;
    }
    CK(cudaMemcpyAsync(c->d.parts + p, &P, sizeof(P), cudaMemcpyHostToDevice, c->stream), "upload particle");
    CK(c->kt->voxelise(c->d, p, P, c->stream), "voxelise");
    c->parts_host[p] = P;
    c->nparts++;
    c->part_cap_host.push_back((int)(18 * side2 * side2 * side2));
    lbve_status s = layout_links(c);
    if (s != LBVE_OK) return s;
    if (id) *id = p;
    return LBVE_OK;
}

lbve_status lbve_read_conversions(lbve_ctx *c, double out[8]) {
    if (!c || !out) return c ? fail(c, LBVE_EINVAL, "out is NULL") : LBVE_EINVAL;
    CK(cudaMemcpyAsync(out, c->pdiag, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream), "read diag");
    CK(cudaStreamSynchronize(c->stream), "read diag sync");
    return LBVE_OK;
}

// ---------------------------------------------------------------------------------
// checkpoint / restore: the raw state of a solve at a step boundary
// ---------------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];  // "LBVECKP1"
    int nx, ny, nz, pdf_prec, nparts, cur, ucur, reserved;
    long long t;
    long long n, np;
    unsigned long long pdf_bytes, real_bytes;
};
static size_t ckpt_bytes(const lbve_ctx *c) {
    const long long np = c->d.g.np, n = c->d.g.n;
    return sizeof(CkptHeader) + (size_t)Q * np * c->kt->pdf_bytes + (size_t)6 * np * c->kt->real_bytes + (size_t)n +
           sizeof(PartDev) * (size_t)c->nparts + sizeof(double) * 8 + sizeof(double) * 256 * 3;
}

size_t lbve_checkpoint_bytes(const lbve_ctx *c) { return c ? ckpt_bytes(c) : 0; }

lbve_status lbve_save(lbve_ctx *c, void *buf, size_t bytes) {
    if (!c) return LBVE_EINVAL;
    if (!buf || bytes < ckpt_bytes(c)) return fail(c, LBVE_EINVAL, "checkpoint buffer missing or too small");
    const long long np = c->d.g.np, n = c->d.g.n;
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBVECKP1", 8);
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.nz = c->p.nz;
    h.pdf_prec = c->p.pdf_prec;
    h.nparts = c->nparts;
    h.cur = c->d.cur;
    h.ucur = c->d.ucur;
    h.t = c->t;
    h.n = n;
    h.np = np;
    h.pdf_bytes = c->kt->pdf_bytes;
    h.real_bytes = c->kt->real_bytes;
    char *o = (char *)buf;
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t fb = (size_t)Q * np * c->kt->pdf_bytes, tb = (size_t)6 * np * c->kt->real_bytes;
    CK(cudaMemcpyAsync(o, c->d.f, fb, cudaMemcpyDeviceToHost, c->stream), "save pdfs");
    o += fb;
    CK(cudaMemcpyAsync(o, c->d.tau[c->d.cur], tb, cudaMemcpyDeviceToHost, c->stream), "save stress");
    o += tb;
    CK(cudaMemcpyAsync(o, c->d.flag, (size_t)n, cudaMemcpyDeviceToHost, c->stream), "save flags");
    o += n;
    if (c->nparts > 0)
        CK(cudaMemcpyAsync(o, c->d.parts, sizeof(PartDev) * c->nparts, cudaMemcpyDeviceToHost, c->stream),
           "save particles");
    o += sizeof(PartDev) * c->nparts;
    CK(cudaMemcpyAsync(o, c->pdiag, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream), "save diag");
    o += sizeof(double) * 8;
    CK(cudaMemcpyAsync(o, c->body_F, sizeof(double) * 256 * 3, cudaMemcpyDeviceToHost, c->stream), "save forces");
    CK(cudaStreamSynchronize(c->stream), "save sync");
    return LBVE_OK;
}

lbve_status lbve_restore(lbve_ctx *c, const void *buf, size_t bytes) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) return fail(c, LBVE_ESTATE, "a pool member cannot be restored");
    if (!buf || bytes < sizeof(CkptHeader)) return fail(c, LBVE_EINVAL, "checkpoint buffer missing or too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "LBVECKP1", 8) != 0) return fail(c, LBVE_EINVAL, "not a checkpoint record");
    if (h.nx != c->p.nx || h.ny != c->p.ny || h.nz != c->p.nz || h.pdf_prec != c->p.pdf_prec ||
        h.np != c->d.g.np || h.pdf_bytes != c->kt->pdf_bytes || h.real_bytes != c->kt->real_bytes)
        return fail(c, LBVE_EINVAL, "checkpoint of a different grid or precision");
    if (h.nparts != c->nparts) return fail(c, LBVE_EINVAL, "checkpoint has a different number of particles");
    if (bytes < ckpt_bytes(c) || h.t < 0 || (h.cur & ~1) || (h.ucur & ~1))
        return fail(c, LBVE_EINVAL, "checkpoint record truncated or inconsistent");
    const long long np = c->d.g.np, n = c->d.g.n;
    const size_t fb = (size_t)Q * np * c->kt->pdf_bytes, tb = (size_t)6 * np * c->kt->real_bytes;
    const char *in = (const char *)buf + sizeof h;
    const uint8_t *flags = (const uint8_t *)(in + fb + tb);
    // the static geometry (no-slip cells and wall classes) must be the context's own: its
    // wall links were built from it; only fluid and particle cells may differ
    {
        std::vector<uint8_t> mine((size_t)n);
        CK(cudaMemcpyAsync(mine.data(), c->d.flag, (size_t)n, cudaMemcpyDeviceToHost, c->stream), "read flags");
        CK(cudaStreamSynchronize(c->stream), "read flags sync");
        for (long long r = 0; r < n; ++r) {
            const bool sa = mine[r] != FLAG_FLUID && mine[r] < FLAG_PART0;
            const bool sb = flags[r] != FLAG_FLUID && flags[r] < FLAG_PART0;
            if (sa != sb || (sa && mine[r] != flags[r]))
                return fail(c, LBVE_EINVAL, "checkpoint geometry differs from the context's (cell " +
                                                std::to_string(r) + ")");
            if (flags[r] >= FLAG_PART0 && flags[r] - FLAG_PART0 >= c->nparts)
                return fail(c, LBVE_EINVAL, "checkpoint flags name a particle the context does not have");
        }
    }
    c->d.cur = h.cur;
    c->d.ucur = h.ucur;
    CK(cudaMemcpyAsync(c->d.f, in, fb, cudaMemcpyHostToDevice, c->stream), "restore pdfs");
    CK(cudaMemcpyAsync(c->d.tau[c->d.cur], in + fb, tb, cudaMemcpyHostToDevice, c->stream), "restore stress");
    CK(cudaMemcpyAsync(c->d.flag, flags, (size_t)n, cudaMemcpyHostToDevice, c->stream), "restore flags");
    const char *rest = in + fb + tb + n;
    std::vector<PartDev> parts((size_t)c->nparts);
    if (c->nparts > 0) {
        std::memcpy(parts.data(), rest, sizeof(PartDev) * c->nparts);
        for (auto &P : parts) P.changed = 1;  // rebuild every particle's links below
        CK(cudaMemcpyAsync(c->d.parts, parts.data(), sizeof(PartDev) * c->nparts, cudaMemcpyHostToDevice, c->stream),
           "restore particles");
    }
    rest += sizeof(PartDev) * c->nparts;
    CK(cudaMemcpyAsync(c->pdiag, rest, sizeof(double) * 8, cudaMemcpyHostToDevice, c->stream), "restore diag");
    rest += sizeof(double) * 8;
    CK(cudaMemcpyAsync(c->body_F, rest, sizeof(double) * 256 * 3, cudaMemcpyHostToDevice, c->stream),
       "restore forces");
    CK(c->kt->build_mask(c->d, 0, 0, 0, c->p.nx, c->p.ny, c->p.nz, c->stream), "neighbour masks");
    if (c->nparts > 0)
        CK(c->kt->particle_links(c->d, c->nparts, c->links, c->seg_begin, c->seg_count, (int)c->wall_seg_begin.size(),
                                 c->part_cap, c->stream),
           "particle links");
    CK(cudaStreamSynchronize(c->stream), "restore sync");
    for (int p = 0; p < c->nparts; ++p) {
        c->parts_host[p] = parts[p];
        c->parts_host[p].changed = 0;
    }
    c->t = h.t;
    clear_unstable(c);
    return LBVE_OK;
}

// z-planes per block of the fused kernel: enough blocks for several waves over the
// SMs, at least 8 planes so the two recomputed halo planes stay a small overhead.
int fused_zchunk(const lbve_ctx *c) {
    const long long tiles = (long long)((c->p.nx + 31) / 32) * ((c->p.ny + 7) / 8);
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = 12LL * 3 * sms;  // ~12 waves of 3 resident blocks per SM
    long long chunks = (want + tiles - 1) / tiles;
    long long zc = (c->p.nz + chunks - 1) / chunks;
    if (zc < 8) zc = 8;
    if (zc > c->p.nz) zc = c->p.nz;
    return (int)zc;
}

bool use_fused(const lbve_ctx *c, int nsteps) {
    // the split schedule is the measured faster one on GB300; fused on request
    if (c->p.schedule != LBVE_SCHED_FUSED) return false;
    if (c->nbody > 0 || c->nparts > 0) return false;  // forces / fill-drain need the split order
    return nsteps >= 2;
}

lbve_status lbve_step(lbve_ctx *c, int nsteps) {
    if (!c) return LBVE_EINVAL;
    if (nsteps < 0) return fail(c, LBVE_EINVAL, "nsteps must be >= 0");
    if (c->pool) return fail(c, LBVE_ESTATE, "a pool member advances through lbve_pool_step");
    if (c->phase_pending) return fail(c, LBVE_ESTATE, "a stream-collide of lbve_step_phase awaits its stress update");
    if (unstable(c)) return fail(c, flag_status(c), unstable_message(c));
    if (use_fused(c, nsteps)) {
        // stream-collide of the first step, fused (stress of step t-1 + stream-collide of
        // step t) for the others, stress update of the last step
        const int zc = fused_zchunk(c);
        c->d.step = (unsigned)c->t;
        CK(timed_begin(c, LBVE_KT_LB), "timing");
        CK(c->kt->lb(c->d, (int)(c->t & 1), c->stream), "lb kernel");
        CK(timed_end(c), "timing");
        c->t++;
        for (int s = 1; s < nsteps; ++s) {
            c->d.step = (unsigned)c->t;
            CK(timed_begin(c, LBVE_KT_FUSED), "timing");
            CK(c->kt->fused(c->d, (int)(c->t & 1), zc, c->stream), "fused kernel");
            CK(timed_end(c), "timing");
            c->d.cur ^= 1;
            c->d.ucur ^= 1;
            c->t++;
            if (c->ev_used >= 4096) CK(harvest_times(c), "timing harvest");
        }
        CK(timed_begin(c, LBVE_KT_FV), "timing");
        CK(c->kt->fv(c->d, c->stream), "fv kernel");
        CK(timed_end(c), "timing");
        c->d.cur ^= 1;
        return LBVE_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        const int parity = (int)(c->t & 1);
        c->d.step = (unsigned)c->t;
        if (c->nbody > 0) {
            CK(timed_begin(c, LBVE_KT_ME), "timing");
            CK(c->kt->momentum_exchange(c->d, parity, c->links, c->seg_begin, c->seg_count, c->nbody, c->max_seg_len,
                                        c->contrib, c->stream),
               "momentum exchange");
            CK(body_sums(c, c->d.parts, c->stream), "body sums");
            CK(timed_end(c), "timing");
        }
        CK(timed_begin(c, LBVE_KT_LB), "timing");
        CK(c->kt->lb(c->d, parity, c->stream), "lb kernel");
        CK(timed_end(c), "timing");
        c->last_lb_parity = parity;
        CK(timed_begin(c, LBVE_KT_FV), "timing");
        CK(c->kt->fv(c->d, c->stream), "fv kernel");
        CK(timed_end(c), "timing");
        c->d.cur ^= 1;
        if (c->nparts > 0) {
            CK(timed_begin(c, LBVE_KT_PARTICLE), "timing");
            CK(c->kt->particle_update(c->d, c->nparts, c->stream), "particle update");
            CK(c->kt->fill_drain(c->d, parity ^ 1, c->nparts, c->pkind, c->pnf, c->pdelta, c->pconv, c->pdiag, c->stream),
               "fill/drain");
            CK(c->kt->particle_links(c->d, c->nparts, c->links, c->seg_begin, c->seg_count,
                                     (int)c->wall_seg_begin.size(), c->part_cap, c->stream),
               "particle links");
            CK(timed_end(c), "timing");
        }
        c->t++;
        if (c->ev_used >= 4096) CK(harvest_times(c), "timing harvest");
    }
    return LBVE_OK;
}

// ---------------------------------------------------------------------------------
// z-slab decomposition of one domain (halo exchange by the caller)
// ---------------------------------------------------------------------------------
lbve_status lbve_set_z_range(lbve_ctx *c, int z_lo, int z_hi, int z_origin) {
    if (!c) return LBVE_EINVAL;
    if (c->geometry_set || c->nparts > 0) return fail(c, LBVE_ESTATE, "the z range is set before lbve_set_geometry");
    if (c->pool) return fail(c, LBVE_ESTATE, "a pool member cannot become a z-slab");
    if (c->p.periodic[2]) return fail(c, LBVE_EINVAL, "a z-slab is not periodic in z: its ghost planes hold the neighbours");
    if (!(z_lo >= 1 && z_lo < z_hi && z_hi <= c->p.nz - 1))
        return fail(c, LBVE_EINVAL, "the computed planes need one ghost plane on each side: 1 <= z_lo < z_hi <= nz - 1");
    if (c->p.schedule == LBVE_SCHED_FUSED) return fail(c, LBVE_EINVAL, "z-slabs run on the split schedule");
    if (z_origin < 0) return fail(c, LBVE_EINVAL, "z_origin must be >= 0");
    c->d.zlo = z_lo;
    c->d.zhi = z_hi;
    // global index of local cell r: r + (z_origin - z_lo) nx ny (modulo 2^32, as the keys)
    c->d.key_base = (unsigned)((long long)(z_origin - z_lo) * c->p.nx * c->p.ny);
    return LBVE_OK;
}

lbve_status lbve_step_phase(lbve_ctx *c, int phase) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) return fail(c, LBVE_ESTATE, "a pool member advances through lbve_pool_step");
    if (phase == 0) {
        if (c->phase_pending) return fail(c, LBVE_ESTATE, "phase 0 twice: the stress update of the last one is missing");
        if (unstable(c)) return fail(c, flag_status(c), unstable_message(c));
        const int parity = (int)(c->t & 1);
        c->d.step = (unsigned)c->t;
        if (c->nbody > 0) {
            CK(c->kt->momentum_exchange(c->d, parity, c->links, c->seg_begin, c->seg_count, c->nbody, c->max_seg_len,
                                        c->contrib, c->stream),
               "momentum exchange");
            CK(body_sums(c, c->d.parts, c->stream), "body sums");
        }
        CK(c->kt->lb(c->d, parity, c->stream), "lb kernel");
        c->last_lb_parity = parity;
        c->phase_pending = true;
        return LBVE_OK;
    }
    if (phase == 1) {
        if (!c->phase_pending) return fail(c, LBVE_ESTATE, "phase 1 without the stream-collide of phase 0");
        CK(c->kt->fv(c->d, c->stream), "fv kernel");
        c->d.cur ^= 1;
        c->t++;
        c->phase_pending = false;
        return LBVE_OK;
    }
    return fail(c, LBVE_EINVAL, "phase must be 0 or 1");
}

size_t lbve_halo_bytes(const lbve_ctx *c, int what) {
    if (!c || what < LBVE_HALO_F || what > LBVE_HALO_TAU) return 0;
    const size_t plane = (size_t)c->p.nx * (size_t)c->p.ny;
    const size_t values = what == LBVE_HALO_F ? 5 : (what == LBVE_HALO_U ? 3 : 6);  // PDFs crossing a face, u, tau
    return plane * values * (what == LBVE_HALO_F ? c->kt->pdf_bytes : c->kt->real_bytes);
}

static lbve_status halo_check(lbve_ctx *c, int what, int side, const void *buf) {
    if (c->d.zhi <= 0) return fail(c, LBVE_ESTATE, "not a z-slab (lbve_set_z_range)");
    if (what < LBVE_HALO_F || what > LBVE_HALO_TAU) return fail(c, LBVE_EINVAL, "unknown halo field");
    if (side != 0 && side != 1) return fail(c, LBVE_EINVAL, "side must be 0 (low z) or 1 (high z)");
    if (!buf) return fail(c, LBVE_EINVAL, "halo buffer is NULL");
    return LBVE_OK;
}

lbve_status lbve_halo_pack(lbve_ctx *c, int what, int side, void *dev_buf) {
    if (!c) return LBVE_EINVAL;
    lbve_status s = halo_check(c, what, side, dev_buf);
    if (s != LBVE_OK) return s;
    CK(c->kt->halo_pack(c->d, what, side, c->last_lb_parity, dev_buf, c->stream), "halo pack");
    return LBVE_OK;
}

lbve_status lbve_halo_unpack(lbve_ctx *c, int what, int side, const void *dev_buf) {
    if (!c) return LBVE_EINVAL;
    lbve_status s = halo_check(c, what, side, dev_buf);
    if (s != LBVE_OK) return s;
    CK(c->kt->halo_unpack(c->d, what, side, c->last_lb_parity, dev_buf, c->stream), "halo unpack");
    return LBVE_OK;
}

lbve_status lbve_read_fields_device(lbve_ctx *c, double *rho, double *u, double *tau) {
    if (!c) return LBVE_EINVAL;
    CK(c->kt->read(c->d, (int)(c->t & 1), rho, u, tau, 0, c->p.nz, c->d.g.n, c->stream), "read kernel");
    return LBVE_OK;
}

lbve_status lbve_read_fields(lbve_ctx *c, double *rho, double *u, double *tau, uint8_t *flags) {
    if (!c) return LBVE_EINVAL;
    const long long n = c->d.g.n, plane = (long long)c->p.nx * c->p.ny;
    double *drho = rho ? (double *)mapped_host(rho) : nullptr;
    double *du = u ? (double *)mapped_host(u) : nullptr;
    double *dtau = tau ? (double *)mapped_host(tau) : nullptr;
    if ((rho || u || tau) && (!rho || drho) && (!u || du) && (!tau || dtau)) {
        // page-locked buffers the device can address: one kernel writes them in place
        CK(c->kt->read(c->d, (int)(c->t & 1), drho, du, dtau, 0, c->p.nz, n, c->stream), "read kernel");
    } else if (rho || u || tau) {
        const int zs = slab_planes(c);
        const long long cap = plane * zs;
        double *st = (double *)dev_alloc(c, sizeof(double) * 10 * (size_t)cap);
        if (!st) return fail(c, LBVE_ENOMEM, "read staging allocation failed");
        prefault_output(rho, sizeof(double) * (size_t)n);
        prefault_output(u, sizeof(double) * 3 * (size_t)n);
        prefault_output(tau, sizeof(double) * 6 * (size_t)n);
        for (int z0 = 0; z0 < c->p.nz; z0 += zs) {
            const int z1 = std::min(c->p.nz, z0 + zs);
            const long long r0 = (long long)z0 * plane, cnt = (long long)(z1 - z0) * plane;
            double *srho = st, *su = st + cnt, *stau = st + 4 * cnt;
            CK(c->kt->read(c->d, (int)(c->t & 1), rho ? srho : nullptr, u ? su : nullptr, tau ? stau : nullptr, z0, z1,
                           cnt, c->stream),
               "read kernel");
            if (rho) CK(cudaMemcpyAsync(rho + r0, srho, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream), "read rho");
            for (int k = 0; u && k < 3; ++k)
                CK(cudaMemcpyAsync(u + k * n + r0, su + k * cnt, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream),
                   "read u");
            for (int k = 0; tau && k < 6; ++k)
                CK(cudaMemcpyAsync(tau + k * n + r0, stau + k * cnt, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                                   c->stream),
                   "read tau");
        }
        CK(cudaStreamSynchronize(c->stream), "read sync");
        dev_free(c, st);
    }
    if (flags) {
        prefault_output(flags, (size_t)n);
        CK(cudaMemcpyAsync(flags, c->d.flag, (size_t)n, cudaMemcpyDeviceToHost, c->stream), "read flags");
    }
    CK(cudaStreamSynchronize(c->stream), "read sync");
    return LBVE_OK;
}

lbve_status lbve_read_pdfs(lbve_ctx *c, double *f) {
    if (!c || !f) return c ? fail(c, LBVE_EINVAL, "f is NULL") : LBVE_EINVAL;
    const long long n = c->d.g.n;
    double *d = (double *)dev_alloc(c, sizeof(double) * Q * n);
    if (!d) return fail(c, LBVE_ENOMEM, "pdf staging allocation failed");
    CK(c->kt->pdfs_io(c->d, (int)(c->t & 1), d, 0, c->stream), "pdf read kernel");
    prefault_output(f, sizeof(double) * Q * (size_t)n);
    CK(cudaMemcpyAsync(f, d, sizeof(double) * Q * n, cudaMemcpyDeviceToHost, c->stream), "pdf copy");
    CK(cudaStreamSynchronize(c->stream), "pdf sync");
    dev_free(c, d);
    return LBVE_OK;
}

lbve_status lbve_write_pdfs(lbve_ctx *c, const double *f) {
    if (!c || !f) return c ? fail(c, LBVE_EINVAL, "f is NULL") : LBVE_EINVAL;
    const long long n = c->d.g.n;
    double *d = (double *)dev_alloc(c, sizeof(double) * Q * n);
    if (!d) return fail(c, LBVE_ENOMEM, "pdf staging allocation failed");
    CK(cudaMemcpyAsync(d, f, sizeof(double) * Q * n, cudaMemcpyHostToDevice, c->stream), "pdf copy");
    CK(c->kt->pdfs_io(c->d, (int)(c->t & 1), d, 1, c->stream), "pdf write kernel");
    CK(cudaStreamSynchronize(c->stream), "pdf sync");
    dev_free(c, d);
    clear_unstable(c);
    return LBVE_OK;
}

lbve_status lbve_read_particle(lbve_ctx *c, int id, double out[24]) {
    if (!c) return LBVE_EINVAL;
    if (id < 0 || id >= c->nparts || !out) return fail(c, LBVE_EINVAL, "no such particle");
    PartDev P;
    CK(cudaMemcpyAsync(&P, c->d.parts + id, sizeof(PartDev), cudaMemcpyDeviceToHost, c->stream), "read particle");
    CK(cudaStreamSynchronize(c->stream), "read particle sync");
    for (int a = 0; a < 3; ++a) {
        out[a] = P.X[a];
        out[3 + a] = P.v[a];
        out[6 + a] = P.w[a];
        out[9 + a] = P.Fme[a];
        out[12 + a] = P.Tme[a];
        out[15 + a] = P.dP[a];
        out[18 + a] = P.dL[a];
    }
    out[21] = P.m;
    out[22] = P.I;
    out[23] = P.R;
    return LBVE_OK;
}

lbve_status lbve_read_body_forces(lbve_ctx *c, double *out) {
    if (!c || !out) return c ? fail(c, LBVE_EINVAL, "out is NULL") : LBVE_EINVAL;
    CK(cudaMemcpyAsync(out, c->body_F, sizeof(double) * 256 * 3, cudaMemcpyDeviceToHost, c->stream), "read forces");
    CK(cudaStreamSynchronize(c->stream), "read forces sync");
    return LBVE_OK;
}

lbve_status lbve_reduce(lbve_ctx *c, double out[6]) {
    if (!c || !out) return c ? fail(c, LBVE_EINVAL, "out is NULL") : LBVE_EINVAL;
    long long nb = 0;
    c->kt->reduce(c->d, 0, nullptr, &nb, c->stream);
    if ((size_t)nb * 6 > c->red_cap) {
        dev_free(c, c->red);
        c->red = (double *)dev_alloc(c, sizeof(double) * 6 * (size_t)nb);
        if (!c->red) return fail(c, LBVE_ENOMEM, "reduction scratch allocation failed");
        c->red_cap = (size_t)nb * 6;
    }
    CK(c->kt->reduce(c->d, (int)(c->t & 1), c->red, &nb, c->stream), "reduce kernel");
    k_final_sum<<<1, 256, 0, c->stream>>>(c->red, nb, c->red_out);
    CK(cudaGetLastError(), "final sum");
    CK(cudaMemcpyAsync(out, c->red_out, sizeof(double) * 6, cudaMemcpyDeviceToHost, c->stream), "reduce copy");
    CK(cudaStreamSynchronize(c->stream), "reduce sync");
    return LBVE_OK;
}

lbve_status lbve_set_kernel_timing(lbve_ctx *c, int enable) {
    if (!c) return LBVE_EINVAL;
    CK(harvest_times(c), "timing harvest");
    c->timing = enable != 0;
    for (int k = 0; k < LBVE_KT_COUNT; ++k) {
        c->kt_ms[k] = 0.0;
        c->kt_count[k] = 0;
    }
    return LBVE_OK;
}

lbve_status lbve_read_kernel_times(lbve_ctx *c, double ms[LBVE_KT_COUNT], long long launches[LBVE_KT_COUNT]) {
    if (!c || !ms || !launches) return c ? fail(c, LBVE_EINVAL, "NULL output") : LBVE_EINVAL;
    CK(harvest_times(c), "timing harvest");
    for (int k = 0; k < LBVE_KT_COUNT; ++k) {
        ms[k] = c->kt_ms[k];
        launches[k] = c->kt_count[k];
    }
    return LBVE_OK;
}

// Fixed reduction shape of a solve's residual (depends only on its size).
static int residual_blocks(const lbve_ctx *c) {
    long long b = (c->d.g.n + 255) / 256;
    return (int)(b > 1024 ? 1024 : (b < 1 ? 1 : b));
}

static lbve_status residual_enqueue(lbve_ctx *c) {
    const int nb = residual_blocks(c);
    if (!c->usnap) {
        c->usnap = dev_alloc(c, (size_t)3 * c->d.g.np * c->kt->real_bytes);
        c->res_partial = (double *)dev_alloc(c, sizeof(double) * 2 * 1024);
        if (!c->usnap || !c->res_partial) return fail(c, LBVE_ENOMEM, "residual buffers");
        CK(cudaMemsetAsync(c->usnap, 0, (size_t)3 * c->d.g.np * c->kt->real_bytes, c->stream), "residual clear");
    }
    CK(c->kt->residual(c->d, c->usnap, c->res_partial, nb, c->stream), "residual kernel");
    return LBVE_OK;
}

static void residual_finish(const lbve_ctx *c, const double *partial, double out[2]) {
    double d2 = 0.0, u2 = 0.0;
    const int nb = residual_blocks(c);
    for (int b = 0; b < nb; ++b) {
        d2 += partial[2 * b];
        u2 += partial[2 * b + 1];
    }
    out[1] = std::sqrt(u2);
    out[0] = u2 > 0.0 ? std::sqrt(d2) / out[1] : (d2 > 0.0 ? INFINITY : 0.0);
}

lbve_status lbve_residual(lbve_ctx *c, double out[2]) {
    if (!c || !out) return c ? fail(c, LBVE_EINVAL, "out is NULL") : LBVE_EINVAL;
    lbve_status s = residual_enqueue(c);
    if (s != LBVE_OK) return s;
    std::vector<double> h(2 * 1024);
    CK(cudaMemcpyAsync(h.data(), c->res_partial, sizeof(double) * 2 * residual_blocks(c), cudaMemcpyDeviceToHost,
                       c->stream),
       "residual copy");
    CK(cudaStreamSynchronize(c->stream), "residual sync");
    residual_finish(c, h.data(), out);
    return LBVE_OK;
}

long long lbve_time(const lbve_ctx *c) { return c ? c->t : -1; }

lbve_status lbve_synchronize(lbve_ctx *c) {
    if (!c) return LBVE_EINVAL;
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    if (unstable(c)) return fail(c, flag_status(c), unstable_message(c));
    return LBVE_OK;
}

int lbve_is_unstable(const lbve_ctx *c) { return c ? (unstable(c) ? 1 : 0) : -1; }

int lbve_stream_collide_kernel(const lbve_ctx *c) {
    if (!c) return -1;
    return c->kt->lb_rows_used(c->d) ? LBVE_LB_ROWS : LBVE_LB_CELLS;
}

int lbve_stress_kernel(const lbve_ctx *c) {
    if (!c) return -1;
    return c->kt->fv_pair_used(c->d) ? LBVE_FV_PAIRS : LBVE_FV_TILES;
}

const char *lbve_last_error(const lbve_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char *lbve_status_string(lbve_status s) {
    return (s >= 0 && s <= LBVE_ESTATE) ? kStatusNames[s] : "LBVE_UNKNOWN";
}

} // extern "C"

// ---------------------------------------------------------------------------------
// pools: resident solves stepped together by the batched persistent kernels
// ---------------------------------------------------------------------------------
struct lbve_pool {
    int prec = 0;
    size_t budget = 0, in_use = 0;
    cudaStream_t stream = nullptr;
    const KernelTable *kt = nullptr;
    std::vector<lbve_ctx *> members;
    std::vector<size_t> member_bytes;
    std::string err;
    // packed work lists, built from the members' state when the membership changes; a step
    // k after the build swaps the stress ping-pong and the AA parity k times.  entries[0]:
    // the members grouped by stress tile width (one stress launch per group); entries[1]:
    // the members grouped by their AA parity at the build (one stream-collide launch per
    // group, lb_class[p] = {first entry, entries, work items} of the group of parity p)
    void *entries[2] = {nullptr, nullptr};
    struct LbClass {
        int start = 0, n = 0, total = 0;
    };
    LbClass lb_class[2];
    size_t entries_cap = 0;
    // particle-phase entries of the members with particles (one block each per step)
    void *pentries = nullptr;
    size_t pentries_cap = 0;
    int n_pentries = 0;
    int total_lb = 0;
    int grid_lb = 0;
    unsigned *dstep = nullptr;  // device: steps since the entries were built
    struct FvGroup {
        int tx, start, n, total, grid;  // stress tile width, first entry, entries, items, grid
        int var;                        // 1 when a member of the group uses a finite-volume variant
    };
    std::vector<FvGroup> fv_groups;
    bool dirty = true;
    long long steps_since_build = 0;
    // residual staging
    double *res_dev = nullptr;
    size_t res_cap = 0;
    // CUDA graphs, one per call parity
    bool use_graphs = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps[2] = {0, 0};
    // side streams: the members' small per-step kernels (momentum exchange, body sums,
    // particle update, fill/drain, links) touch only their own buffers, so the chains of
    // different members run side by side, forked from and joined back to the pool stream
    // (in a captured graph, one branch per side stream: 64 measured 6 % faster per pool
    // step than 8 on a 48-member mix, 32 5 %)
    static constexpr int kSide = 64;
    cudaStream_t side[kSide] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
    bool side_ready = false;
};

namespace {

lbve_status pfail(lbve_pool *P, lbve_status s, const std::string &m) {
    if (P) P->err = m;
    return s;
}

#define PCK(call, where)                                                                           \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return pfail(P, LBVE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void drop_graphs(lbve_pool *P) {
    for (int k = 0; k < 2; ++k) {
        if (P->graph[k]) cudaGraphExecDestroy(P->graph[k]);
        P->graph[k] = nullptr;
        P->graph_steps[k] = 0;
    }
}

// Entries for the two parities of the call (state after an even / odd number of steps
// since the build), uploaded once per membership change.
lbve_status build_entries(lbve_pool *P) {
    const size_t eb = P->kt->batch_entry_bytes;
    const size_t n = P->members.size();
    if (n > P->entries_cap) {
        for (int k = 0; k < 2; ++k) {
            if (P->entries[k]) cudaFree(P->entries[k]);
            P->entries[k] = nullptr;
            PCK(cudaMalloc(&P->entries[k], eb * std::max<size_t>(n, 16)), "pool entries");
        }
        P->entries_cap = std::max<size_t>(n, 16);
    }
    // entries grouped by stress tile width (one stress launch per group); the stream-collide
    // numbers its items over all entries
    std::vector<unsigned char> host(eb * std::max<size_t>(n, 1));
    P->fv_groups.clear();
    int lb_first = 0;
    size_t slot = 0;
    for (int tx : {16, 32, 64}) {
        lbve_pool::FvGroup grp{tx, (int)slot, 0, 0, 0, 0};
        int fv_first = 0;
        for (size_t m = 0; m < n; ++m) {
            const lbve_ctx *c = P->members[m];
            int lbe = 0, fve = 0;
            P->kt->batch_tiles(c->d, c->lb_tx, c->fv_tx, &lbe, &fve);
            if (fve != tx) continue;
            const int parity = (int)(c->t & 1);
            DevState d = c->d;
            d.step = (unsigned)c->t;  // step k of a launch sequence performs step t + k
            int lbi = 0, fvi = 0;
            P->kt->fill_entry(d, parity, lb_first, fv_first, 0, lbe, fve, host.data() + eb * slot, &lbi, &fvi);
            lb_first += lbi;
            fv_first += fvi;
            ++slot;
            ++grp.n;
            grp.var |= P->kt->fv_variant_of(c->d);
        }
        if (grp.n == 0) continue;
        grp.total = fv_first;
        grp.grid = P->kt->batched_grid(tx);
        P->fv_groups.push_back(grp);
    }
    if (slot != n) return pfail(P, LBVE_ECUDA, "internal: stress tile of a member not covered");
    P->total_lb = lb_first;
    if (n) PCK(cudaMemcpyAsync(P->entries[0], host.data(), eb * n, cudaMemcpyHostToDevice, P->stream), "upload entries");
    // stream-collide lists: the members by AA parity at the build, items numbered per list
    std::vector<unsigned char> host_lb(eb * std::max<size_t>(n, 1));
    slot = 0;
    for (int par = 0; par < 2; ++par) {
        lbve_pool::LbClass &cl = P->lb_class[par];
        cl.start = (int)slot;
        cl.n = 0;
        int first = 0;
        for (size_t m = 0; m < n; ++m) {
            const lbve_ctx *c = P->members[m];
            if ((int)(c->t & 1) != par) continue;
            DevState d = c->d;
            d.step = (unsigned)c->t;
            int lbi = 0, fvi = 0;
            P->kt->fill_entry(d, par, first, 0, 0, c->lb_tx, c->fv_tx, host_lb.data() + eb * slot, &lbi, &fvi);
            first += lbi;
            ++slot;
            ++cl.n;
        }
        cl.total = first;
    }
    if (n) PCK(cudaMemcpyAsync(P->entries[1], host_lb.data(), eb * n, cudaMemcpyHostToDevice, P->stream),
               "upload stream-collide entries");
    // particle-phase entries, in member order
    const size_t pb = P->kt->part_entry_bytes;
    std::vector<unsigned char> phost;
    int np_ = 0;
    for (lbve_ctx *c : P->members) {
        if (c->nparts <= 0) continue;
        phost.resize(pb * (size_t)(np_ + 1));
        PartScratch ps;
        ps.nparts = c->nparts;
        ps.first_seg = (int)c->wall_seg_begin.size();
        ps.kind = c->pkind;
        ps.nf = c->pnf;
        ps.delta = c->pdelta;
        ps.diag = c->pdiag;
        ps.conv = c->pconv;
        ps.links = c->links;
        ps.seg_begin = c->seg_begin;
        ps.seg_count = c->seg_count;
        ps.capacity = c->part_cap;
        P->kt->fill_part_entry(c->d, (int)((c->t + 1) & 1), ps, phost.data() + pb * (size_t)np_);
        ++np_;
    }
    if ((size_t)np_ > P->pentries_cap) {
        if (P->pentries) cudaFree(P->pentries);
        P->pentries = nullptr;
        P->pentries_cap = std::max<size_t>((size_t)np_, 16);
        PCK(cudaMalloc(&P->pentries, pb * P->pentries_cap), "pool particle entries");
    }
    P->n_pentries = np_;
    if (np_) PCK(cudaMemcpyAsync(P->pentries, phost.data(), pb * (size_t)np_, cudaMemcpyHostToDevice, P->stream),
                 "upload particle entries");
    PCK(cudaMemsetAsync(P->dstep, 0, sizeof(unsigned), P->stream), "step counter reset");
    PCK(cudaStreamSynchronize(P->stream), "entries sync");
    if (!P->grid_lb) P->grid_lb = P->kt->batched_grid(0);
    P->dirty = false;
    P->steps_since_build = 0;
    drop_graphs(P);
    return LBVE_OK;
}

lbve_status ensure_side_streams(lbve_pool *P) {
    if (P->side_ready) return LBVE_OK;
    PCK(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming), "side event");
    for (int j = 0; j < lbve_pool::kSide; ++j) {
        PCK(cudaStreamCreateWithFlags(&P->side[j], cudaStreamNonBlocking), "side stream");
        PCK(cudaEventCreateWithFlags(&P->ev_join[j], cudaEventDisableTiming), "side event");
    }
    P->side_ready = true;
    return LBVE_OK;
}

// Run body(member, stream) for every listed member: on the pool stream when there is one
// member, else spread over the side streams between a fork and a join on the pool stream.
template <class Body>
lbve_status fan_out(lbve_pool *P, const std::vector<lbve_ctx *> &list, Body &&body) {
    const int ns = std::min<int>(lbve_pool::kSide, (int)list.size());
    if (ns <= 1 || !P->side_ready) {
        for (lbve_ctx *c : list) {
            lbve_status s = body(c, P->stream);
            if (s != LBVE_OK) return s;
        }
        return LBVE_OK;
    }
    PCK(cudaEventRecord(P->ev_fork, P->stream), "fork");
    for (int j = 0; j < ns; ++j) PCK(cudaStreamWaitEvent(P->side[j], P->ev_fork, 0), "fork wait");
    for (size_t i = 0; i < list.size(); ++i) {
        lbve_status s = body(list[i], P->side[i % ns]);
        if (s != LBVE_OK) return s;
    }
    for (int j = 0; j < ns; ++j) {
        PCK(cudaEventRecord(P->ev_join[j], P->side[j]), "join");
        PCK(cudaStreamWaitEvent(P->stream, P->ev_join[j], 0), "join wait");
    }
    return LBVE_OK;
}

// Enqueue nsteps steps of every member on the pool stream (graph-capturable).
lbve_status enqueue_steps(lbve_pool *P, int q, int nsteps) {
    const int n = (int)P->members.size();
    std::vector<lbve_ctx *> with_bodies, with_parts;
    for (lbve_ctx *c : P->members) {
        if (c->nbody > 0) with_bodies.push_back(c);
        if (c->nparts > 0) with_parts.push_back(c);
    }
    for (int k = 0; k < nsteps; ++k) {
        const int kk = q + k;  // steps since the entries were built (they encode that state)
        lbve_status s = fan_out(P, with_bodies, [&](lbve_ctx *c, cudaStream_t st) -> lbve_status {
            DevState d = c->d;  // the member's state at the start of this call
            if (k & 1) d.cur ^= 1;
            const int parity = (int)((c->t + k) & 1);
            PCK(c->kt->momentum_exchange(d, parity, c->links, c->seg_begin, c->seg_count, c->nbody, c->max_seg_len,
                                         c->contrib, st),
                "pool momentum exchange");
            PCK(body_sums(c, d.parts, st), "pool body sums");
            return LBVE_OK;
        });
        if (s != LBVE_OK) return s;
        for (int par = 0; par < 2; ++par) {  // the group of build parity par is at parity (par + kk) & 1
            const lbve_pool::LbClass &cl = P->lb_class[par];
            if (cl.n == 0) continue;
            PCK(P->kt->lb_batched((const unsigned char *)P->entries[1] + (size_t)cl.start * P->kt->batch_entry_bytes,
                                  cl.n, cl.total, kk, P->grid_lb, P->dstep, (par + kk) & 1, P->stream),
                "batched lb");
        }
        k_step_count<<<1, 1, 0, P->stream>>>(P->dstep);
        PCK(cudaGetLastError(), "step counter");
        for (const lbve_pool::FvGroup &grp : P->fv_groups)
            PCK(P->kt->fv_batched((const unsigned char *)P->entries[0] + (size_t)grp.start * P->kt->batch_entry_bytes,
                                  grp.n, grp.total, kk, grp.grid, grp.tx, grp.var, P->stream),
                "batched fv");
        // particle update, fill/drain and links of every member with particles: one block
        // per member in one launch
        if (!with_parts.empty())
            PCK(P->kt->particle_phase_batched(P->pentries, P->n_pentries, kk, P->stream), "pool particle phase");
    }
    return LBVE_OK;
}

} // namespace

extern "C" {

lbve_status lbve_pool_create(int pdf_prec, size_t budget_bytes, void *cuda_stream, lbve_pool **out) {
    if (!out) return LBVE_EINVAL;
    *out = nullptr;
    const KernelTable *kt = table_for(pdf_prec);
    if (!kt) return LBVE_EINVAL;
    lbve_pool *P = new (std::nothrow) lbve_pool();
    if (!P) return LBVE_ENOMEM;
    P->prec = pdf_prec;
    P->budget = budget_bytes;
    P->stream = (cudaStream_t)cuda_stream;
    P->kt = kt;
    if (cudaMalloc(&P->dstep, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return LBVE_ENOMEM;
    }
    *out = P;
    return LBVE_OK;
}

lbve_status lbve_pool_destroy(lbve_pool *P) {
    if (!P) return LBVE_EINVAL;
    cudaStreamSynchronize(P->stream);
    drop_graphs(P);
    if (P->side_ready) {
        for (int j = 0; j < lbve_pool::kSide; ++j) {
            cudaStreamSynchronize(P->side[j]);
            cudaStreamDestroy(P->side[j]);
            cudaEventDestroy(P->ev_join[j]);
        }
        cudaEventDestroy(P->ev_fork);
    }
    for (int k = 0; k < 2; ++k)
        if (P->entries[k]) cudaFree(P->entries[k]);
    if (P->pentries) cudaFree(P->pentries);
    if (P->res_dev) cudaFree(P->res_dev);
    if (P->dstep) cudaFree(P->dstep);
    for (lbve_ctx *c : P->members) c->pool = nullptr;
    delete P;
    return LBVE_OK;
}

int lbve_pool_fits(const lbve_pool *P, const lbve_params *p) {
    if (!P || !p) return 0;
    const size_t b = lbve_device_bytes(p);
    return b > 0 && P->in_use + b <= P->budget ? 1 : 0;
}

lbve_status lbve_pool_admit(lbve_pool *P, lbve_ctx *c) {
    if (!P || !c) return LBVE_EINVAL;
    if (c->pool) return pfail(P, LBVE_ESTATE, "context already belongs to a pool");
    if (c->p.pdf_prec != P->prec) return pfail(P, LBVE_ESTATE, "precision differs from the pool's");
    if (c->stream != P->stream) return pfail(P, LBVE_ESTATE, "stream differs from the pool's");
    if (c->p.fene_L2 > 0.0) return pfail(P, LBVE_ESTATE, "FENE-P solves advance through lbve_step only");
    if (c->d.zhi > 0) return pfail(P, LBVE_ESTATE, "z-slabs advance through lbve_step / lbve_step_phase only");
    const size_t b = lbve_device_bytes(&c->p);
    if (P->in_use + b > P->budget) return pfail(P, LBVE_ENOMEM, "device-memory budget exhausted");
    if (c->lb_tx == 0 && c->fv_tx == 0) tuned_tiles(P->prec, c->p.nx, c->lb_tx, c->fv_tx);
    P->members.push_back(c);
    P->member_bytes.push_back(b);
    P->in_use += b;
    c->pool = P;
    P->dirty = true;
    return LBVE_OK;
}

lbve_status lbve_pool_remove(lbve_pool *P, lbve_ctx *c) {
    if (!P || !c) return LBVE_EINVAL;
    for (size_t k = 0; k < P->members.size(); ++k) {
        if (P->members[k] != c) continue;
        cudaStreamSynchronize(P->stream);
        P->in_use -= P->member_bytes[k];
        P->members.erase(P->members.begin() + (long)k);
        P->member_bytes.erase(P->member_bytes.begin() + (long)k);
        c->pool = nullptr;
        P->dirty = true;
        return LBVE_OK;
    }
    return pfail(P, LBVE_EINVAL, "not a member");
}

lbve_status lbve_pool_step(lbve_pool *P, int nsteps) {
    if (!P) return LBVE_EINVAL;
    if (nsteps < 0) return pfail(P, LBVE_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0 || P->members.empty()) return LBVE_OK;
    for (size_t k = 0; k < P->members.size(); ++k)
        if (unstable(P->members[k]))
            return pfail(P, flag_status(P->members[k]), "member " + std::to_string(k) + " is unstable (" +
                                                unstable_message(P->members[k]) + "); remove it to continue");
    if (P->dirty) {
        lbve_status s = build_entries(P);
        if (s != LBVE_OK) return s;
    }
    {
        lbve_status s = ensure_side_streams(P);
        if (s != LBVE_OK) return s;
    }
    const int q = (int)(P->steps_since_build & 1);
    // the legacy default stream cannot be captured: launch directly there
    const bool graphs = P->use_graphs && (uintptr_t)P->stream > 1;
    if (graphs) {
        if (!P->graph[q] || P->graph_steps[q] != nsteps) {
            if (P->graph[q]) cudaGraphExecDestroy(P->graph[q]);
            P->graph[q] = nullptr;
            cudaGraph_t g;
            PCK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            lbve_status s = enqueue_steps(P, q, nsteps);
            cudaError_t e = cudaStreamEndCapture(P->stream, &g);
            if (s != LBVE_OK) return s;
            PCK(e, "end capture");
            PCK(cudaGraphInstantiate(&P->graph[q], g, 0), "graph instantiate");
            cudaGraphDestroy(g);
            P->graph_steps[q] = nsteps;
        }
        PCK(cudaGraphLaunch(P->graph[q], P->stream), "graph launch");
    } else {
        lbve_status s = enqueue_steps(P, q, nsteps);
        if (s != LBVE_OK) return s;
    }
    for (lbve_ctx *c : P->members) {
        c->t += nsteps;
        if (nsteps & 1) c->d.cur ^= 1;
    }
    P->steps_since_build += nsteps;
    return LBVE_OK;
}

lbve_status lbve_pool_residuals(lbve_pool *P, double *out) {
    if (!P || !out) return P ? pfail(P, LBVE_EINVAL, "out is NULL") : LBVE_EINVAL;
    const size_t n = P->members.size();
    if (n == 0) return LBVE_OK;
    for (lbve_ctx *c : P->members) {
        lbve_status s = residual_enqueue(c);
        if (s != LBVE_OK) return pfail(P, s, c->err);
    }
    std::vector<double> h(2 * 1024);
    for (size_t m = 0; m < n; ++m) {
        lbve_ctx *c = P->members[m];
        PCK(cudaMemcpyAsync(h.data(), c->res_partial, sizeof(double) * 2 * residual_blocks(c), cudaMemcpyDeviceToHost,
                            P->stream),
            "residual copy");
        PCK(cudaStreamSynchronize(P->stream), "residual sync");
        residual_finish(c, h.data(), out + 2 * m);
    }
    return LBVE_OK;
}

int lbve_pool_size(const lbve_pool *P) { return P ? (int)P->members.size() : 0; }
size_t lbve_pool_bytes_in_use(const lbve_pool *P) { return P ? P->in_use : 0; }
lbve_status lbve_pool_set_graphs(lbve_pool *P, int enable) {
    if (!P) return LBVE_EINVAL;
    cudaStreamSynchronize(P->stream);
    P->use_graphs = enable != 0;
    drop_graphs(P);
    return LBVE_OK;
}
const char *lbve_pool_last_error(const lbve_pool *P) { return P ? P->err.c_str() : "NULL pool"; }

} // extern "C"

// ---------------------------------------------------------------------------------
// schedule autotuning (launch shapes only: results do not depend on them)
// ---------------------------------------------------------------------------------
namespace {

// Device milliseconds per step of `steps` steps on the stream, after `warm` untimed calls
// of `steps` steps (a pool captures one graph per call parity: two warm calls leave both
// captured, so no capture falls in the timed call).
template <class StepFn>
lbve_status time_steps(cudaStream_t st, int steps, int warm, StepFn &&step, double &ms, std::string &err) {
    for (int w = 0; w < warm; ++w) {
        lbve_status s = step(steps);
        if (s != LBVE_OK) return s;
    }
    lbve_status s = LBVE_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        err = "event creation failed";
        return LBVE_ECUDA;
    }
    cudaEventRecord(e0, st);
    s = step(steps);
    cudaEventRecord(e1, st);
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LBVE_OK) return s;
    if (e != cudaSuccess) {
        err = std::string("autotune timing: ") + cudaGetErrorString(e);
        return LBVE_ECUDA;
    }
    ms = (double)t / steps;
    return LBVE_OK;
}

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

} // namespace

extern "C" {

lbve_status lbve_autotune(lbve_ctx *c, int steps, lbve_tuning *out) {
    if (!c) return LBVE_EINVAL;
    if (c->pool) return fail(c, LBVE_ESTATE, "a pool member is tuned through its pool");
    if (c->p.schedule == LBVE_SCHED_FUSED) return fail(c, LBVE_ESTATE, "autotuning covers the split schedule");
    lbve_tuning r{};
    const long long t0 = c->t;
    int bx = 0, zc = 0;
    if (steps <= 0 || tuned_ctx(c->p, bx, zc)) {
        if (tuned_ctx(c->p, bx, zc)) {
            c->d.block_x = bx;
            c->d.fv_zchunk = zc;
        }
        r.block_x = c->d.block_x;
        r.fv_zchunk = c->kt->fv_zchunk_of(c->d);
        if (out) *out = r;
        return LBVE_OK;
    }
    auto step = [&](int n) { return lbve_step(c, n); };
    const int bx0 = c->d.block_x, zc0 = c->d.fv_zchunk;
    DevState probe = c->d;
    probe.fv_zchunk = 0;
    const int h = c->kt->fv_zchunk_of(probe);
    std::vector<int> bxs, zcs;
    for (int b : {32, 64, 128})
        if (b == 32 || b / 2 < c->p.nx) bxs.push_back(b);
    for (int z : {std::max(4, h / 2), h, std::min(c->p.nz, 2 * h)})
        if (std::find(zcs.begin(), zcs.end(), z) == zcs.end()) zcs.push_back(z);
    double ms0 = 0.0;
    lbve_status s = time_steps(c->stream, steps, 1, step, ms0, c->err);
    if (s != LBVE_OK) return s;
    double best = ms0;
    int best_bx = bx0, best_zc = zc0 > 0 ? zc0 : h;
    int count = 1;
    for (int b : bxs) {
        for (int z : zcs) {
            if (b == bx0 && z == (zc0 > 0 ? zc0 : h)) continue;  // the starting schedule, measured above
            c->d.block_x = b;
            c->d.fv_zchunk = z;
            double ms = 0.0;
            s = time_steps(c->stream, steps, 1, step, ms, c->err);
            if (s != LBVE_OK) return s;
            ++count;
            if (ms < best) {
                best = ms;
                best_bx = b;
                best_zc = z;
            }
        }
    }
    c->d.block_x = best_bx;
    c->d.fv_zchunk = best_zc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned_ctx[{c->p.pdf_prec, c->p.nx, c->p.ny, c->p.nz}] = {best_bx, best_zc};
    }
    r.block_x = best_bx;
    r.fv_zchunk = best_zc;
    r.candidates = count;
    r.steps_taken = c->t - t0;
    r.ms_per_step = best;
    r.ms_per_step_default = ms0;
    if (out) *out = r;
    return LBVE_OK;
}

lbve_status lbve_pool_autotune(lbve_pool *P, int steps, int max_classes, int *n_classes, int *class_nx, int *lb_tx,
                               int *fv_tx, double *ms_before, double *ms_after) {
    if (!P) return LBVE_EINVAL;
    if (steps <= 0) return pfail(P, LBVE_EINVAL, "steps must be > 0");
    if (P->members.empty()) return pfail(P, LBVE_ESTATE, "the pool has no members");
    // classes by nx, largest total cells first
    std::map<int, long long> cells;
    for (lbve_ctx *c : P->members) cells[c->p.nx] += (long long)c->p.nx * c->p.ny * c->p.nz;
    std::vector<std::pair<long long, int>> order;
    for (auto &kv : cells) order.push_back({-kv.second, kv.first});
    std::sort(order.begin(), order.end());
    auto step = [&](int n) { return lbve_pool_step(P, n); };
    auto set_class = [&](int nx, int lb, int fv) {
        for (lbve_ctx *c : P->members)
            if (c->p.nx == nx) {
                c->lb_tx = lb;
                c->fv_tx = fv;
            }
        P->dirty = true;
    };
    double base = 0.0;
    lbve_status s = time_steps(P->stream, steps, 2, step, base, P->err);
    if (s != LBVE_OK) return s;
    double best = base;
    std::vector<std::array<int, 3>> chosen;
    for (auto &o : order) {
        const int nx = o.second;
        lbve_ctx *rep = nullptr;
        for (lbve_ctx *c : P->members)
            if (c->p.nx == nx) rep = c;
        int cur_lb = 0, cur_fv = 0;
        P->kt->batch_tiles(rep->d, rep->lb_tx, rep->fv_tx, &cur_lb, &cur_fv);
        const int wmax = std::max(16, std::min(128, pow2_at_least(nx)));
        // stream-collide tile width
        for (int lb : {16, 32, 64, 128}) {
            if (lb > wmax || lb == cur_lb) continue;
            set_class(nx, lb, cur_fv);
            double ms = 0.0;
            s = time_steps(P->stream, steps, 2, step, ms, P->err);
            if (s != LBVE_OK) return s;
            if (ms < best) {
                best = ms;
                cur_lb = lb;
            }
        }
        // stress tile width
        for (int fv : {16, 32, 64}) {
            int e_lb = 0, e_fv = 0;
            P->kt->batch_tiles(rep->d, cur_lb, fv, &e_lb, &e_fv);
            if (e_fv != fv || fv == cur_fv || fv > std::max(16, pow2_at_least(nx))) continue;
            set_class(nx, cur_lb, fv);
            double ms = 0.0;
            s = time_steps(P->stream, steps, 2, step, ms, P->err);
            if (s != LBVE_OK) return s;
            if (ms < best) {
                best = ms;
                cur_fv = fv;
            }
        }
        set_class(nx, cur_lb, cur_fv);
        chosen.push_back({nx, cur_lb, cur_fv});
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned_tiles[{P->prec, nx}] = {cur_lb, cur_fv};
    }
    if (n_classes) *n_classes = (int)chosen.size();
    for (int k = 0; k < (int)chosen.size() && k < max_classes; ++k) {
        if (class_nx) class_nx[k] = chosen[k][0];
        if (lb_tx) lb_tx[k] = chosen[k][1];
        if (fv_tx) fv_tx[k] = chosen[k][2];
    }
    if (ms_before) *ms_before = base;
    if (ms_after) *ms_after = best;
    return LBVE_OK;
}

} // extern "C"

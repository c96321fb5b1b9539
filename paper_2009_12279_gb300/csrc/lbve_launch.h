// lbve_launch.h -- internal interface between the host library (lbve_api.cu) and the
// per-precision kernel translation units: parameter structs passed by value to the
// kernels and a table of host-side launchers per PDF storage type.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbve {

constexpr int Q = 19;
constexpr int FLAG_FLUID = 0;
constexpr int FLAG_NOSLIP = 1;
constexpr int FLAG_WALL0 = 2;
constexpr int MAX_WALL = 16;
constexpr int FLAG_PART0 = 64;
constexpr int MAX_PART = 64;

struct Geo {
    int nx, ny, nz;
    int per[3];
    long long n;  // nx*ny*nz
    long long np; // stride between the arrays of one field (n rounded up to 64)
};

template <class R>
struct Phys {
    R omega_p, omega_m;
    R A, B;        // 3 (1 - omega-/2) and 1 - omega+/2 of the forcing term
    R ep_l, inv_l; // eta_p / lambda_p and 1 / lambda_p
    R g[3];
    R rho0;        // shift base of the stored deviations (0 in FP64 mode)
    R rho_ref;     // reference density rho0 of the solve (all modes)
    R scale, inv_scale;
    int flux_on, src_on;
    int ctu_on;   // face fluxes scaled by the transverse overlap of the displaced donor cell
    int divu_on;  // the tau div(u) source term
    R gk;         // alpha / eta_p of the Giesekus source term (0: Oldroyd-B)
    int fene;     // FENE-P: the stress arrays hold the conformation tensor A
    R fene_L2;    // its maximum extensibility L^2
    R eta_p, lam; // polymer viscosity and relaxation time (stress <-> conformation)
    R wall_vel[MAX_WALL][3];
};

// FP64 rigid-sphere state used by the particle kernels.
struct PartDev {
    double X[3], v[3], w[3];
    double R, rho_p, m, I;
    double Fext[3], Text[3];
    double Fme[3], Tme[3];
    double dP[3], dL[3];
    int changed;  // 1 when the last fill/drain converted cells (links must be rebuilt)
};

// A solve's particle scratch and link arrays, as the particle-phase kernels take them.
struct PartScratch {
    int nparts, first_seg;
    uint8_t *kind, *nf;
    double *delta, *diag;
    int *conv;
    long long *links;
    const int *seg_begin;
    int *seg_count;
    const int *capacity;
};

// Device buffers of one solve.
struct DevState {
    Geo g;
    Phys<double> ph;  // converted to the kernel's real type by the launchers
    void *f;          // 19 * np PDF storage elements
    void *tau[2];     // 6 * np reals each (ping-pong)
    void *u[2];       // 3 * np reals each (velocity of the last stream-collide, ping-pong)
    int ucur;         // index of the velocity written by the last stream-collide
    uint32_t *mask;   // np neighbour masks
    uint8_t *flag;    // np bytes
    PartDev *parts;   // MAX_PART entries
    int cur;          // index of tau^t in tau[]
    int block_x;      // threads per block along x
    int fv_zchunk;    // z-planes per block of the stress kernel (0: by the SM count)
    unsigned step;    // index of the step the next stream-collide performs (low 32 bits)
    // instability flag: a word of mapped page-locked host memory (its device address)
    // that the stream-collide sets to 1 when a fluid cell has rho <= 0, |u|^2 >= 1/3
    // (the lattice sound speed squared) or a NaN; nullptr: no check
    unsigned *bad = nullptr;
    // planes [zlo, zhi) that the step kernels compute (zhi 0: all); the planes outside are
    // the ghost planes of a z-slab of a decomposed domain, filled by the halo exchange
    int zlo = 0, zhi = 0;
    // offset of this grid's cell indices in the decomposed domain's (rounding keys of the
    // 16-bit stores use global cells, so a slab rounds as the undecomposed domain does)
    unsigned key_base = 0;
    // the row-pipelined stream-collide (k_lb_rows) and the two-cell stress kernel
    // (k_fv_pair) where the grid allows them: 0 never (schedule SPLIT), 1 on large grids
    // only (AUTO), 2 always (PIPELINED); else the per-cell stream-collide and the tiled
    // stress kernel.  lb_rows_yc: rows per strip of the row pipeline (0: by the SM count)
    int auto_kernels = 0;
    int lb_rows_yc = 0;
};

struct KernelTable {
    int prec;          // lbve_pdf_prec
    size_t pdf_bytes;  // bytes per stored PDF
    size_t real_bytes; // bytes per stress / velocity value
    cudaError_t (*init)(const DevState &, const double *rho, const double *u, const double *tau, long long r0,
                        long long count, long long ld, cudaStream_t);
    cudaError_t (*lb)(const DevState &, int parity, cudaStream_t);
    cudaError_t (*fv)(const DevState &, cudaStream_t);
    // FP64: 8 doubles per link in contrib; shifted modes: 8 doubles per (segment, block of
    // 128 links), ceil(max_len / 128) blocks per segment
    cudaError_t (*momentum_exchange)(const DevState &, int parity, const long long *links, const int *seg_begin,
                                     const int *seg_count, int nseg, int max_len, double *contrib, cudaStream_t);
    cudaError_t (*voxelise)(const DevState &, int p, const PartDev &host, cudaStream_t);
    cudaError_t (*particle_update)(const DevState &, int nparts, cudaStream_t);
    cudaError_t (*particle_links)(const DevState &, int nparts, long long *links, const int *seg_begin, int *seg_count,
                                  int first_seg, const int *capacity, cudaStream_t);
    cudaError_t (*fill_drain)(const DevState &, int parity, int nparts, uint8_t *kind, uint8_t *nf, double *delta,
                              int *conv, double *diag, cudaStream_t);
    cudaError_t (*read)(const DevState &, int parity, double *rho, double *u, double *tau, int z0, int z1,
                        long long ld, cudaStream_t);
    cudaError_t (*pdfs_io)(const DevState &, int parity, double *io, int write, cudaStream_t);
    cudaError_t (*reduce)(const DevState &, int parity, double *partial, long long *nblocks, cudaStream_t);
    cudaError_t (*probe)(const DevState &, int parity, const long long *cells, int count, double *out, cudaStream_t);
    cudaError_t (*build_mask)(const DevState &, int lx, int ly, int lz, int ex, int ey, int ez, cudaStream_t);
    cudaError_t (*fused)(const DevState &, int parity, int zchunk, cudaStream_t);
    // batched schedule (pools)
    size_t batch_entry_bytes;
    // lb_tx / fv_tx: the solve's tile widths in the batched kernels (0: default by nx)
    void (*fill_entry)(const DevState &, int parity, int lb_first, int fv_first, int fv_zchunk, int lb_tx, int fv_tx,
                       void *entry, int *lb_items, int *fv_items);
    // dstep: device counter of the steps since the entries were built (their step index base)
    cudaError_t (*lb_batched)(const void *entries, int n, int total, int k, int grid, const unsigned *dstep,
                              int parity, cudaStream_t);  // entries all at AA parity `parity` at step k
    // stress update of the solves with stress tile width tx (entries: that group only);
    // var: some solve of the group uses a finite-volume variant
    cudaError_t (*fv_batched)(const void *entries, int n, int total, int k, int grid, int tx, int var, cudaStream_t);
    int (*batched_grid)(int which);  // resident blocks: 0 stream-collide, else stress tile width
    cudaError_t (*residual)(const DevState &, void *usnap, double *partial, int nblocks, cudaStream_t);
    // the tile widths fill_entry will use for requested widths (0: default by nx)
    void (*batch_tiles)(const DevState &, int lb_tx, int fv_tx, int *lb_eff, int *fv_eff);
    int (*fv_zchunk_of)(const DevState &);  // z-planes per block the stress kernel will use
    int (*fv_variant_of)(const DevState &);  // 1 when the solve uses a finite-volume variant
    // pools: the particle phase (update, fill/drain, links) of every member with
    // particles in one launch; entries built per member like the batch entries
    size_t part_entry_bytes;
    void (*fill_part_entry)(const DevState &, int parity0, const PartScratch &, void *entry);
    cudaError_t (*particle_phase_batched)(const void *entries, int n, int k, cudaStream_t);
    // z-slab halo exchange: what 0 PDFs of the last stream-collide (its AA parity), 1 u,
    // 2 tau; side 0 the low z side, 1 the high one; buf a device buffer of plane-major
    // values (halo_values(what) per cell of an x-y plane, storage type for the PDFs)
    cudaError_t (*halo_pack)(const DevState &, int what, int side, int parity, void *buf, cudaStream_t);
    cudaError_t (*halo_unpack)(const DevState &, int what, int side, int parity, const void *buf, cudaStream_t);
    int (*lb_rows_used)(const DevState &);  // 1 when the stream-collide runs the row pipeline
    int (*fv_pair_used)(const DevState &);  // 1 when the stress update runs two cells per thread
};

// Bounding-box side used to size the per-particle scratch (cells within R + margin).
inline int particle_box_side(double R, int margin) {
    int c = (int)R;
    if ((double)c < R) ++c;
    return 2 * c + 2 * margin + 3;
}

const KernelTable *table_f64();
const KernelTable *table_f32();
const KernelTable *table_f16();
const KernelTable *table_bf16();

} // namespace lbve

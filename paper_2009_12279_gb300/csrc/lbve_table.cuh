// lbve_table.cuh -- host-side launchers of the step kernels for one PDF storage type,
// collected in a KernelTable.  Included once per storage type by the precision TUs.
#pragma once

#include <algorithm>
#include <atomic>

#include "lbve_kernels.cuh"
#include "lbve_rows.cuh"

namespace lbve {

// Dynamic shared-memory limit of a kernel raised once per device: the attribute is per
// device, so the record is a bit per device ordinal (idempotent if two threads race).
struct SmemAttrOnce {
    std::atomic<unsigned long long> done[2] = {{0ull}, {0ull}};
    template <class K>
    cudaError_t ensure(K kernel, size_t bytes) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 128) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        const unsigned long long bit = 1ull << (dev & 63);
        std::atomic<unsigned long long> &w = done[dev >> 6];
        if (w.load(std::memory_order_acquire) & bit) return cudaSuccess;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e == cudaSuccess) w.fetch_or(bit, std::memory_order_acq_rel);
        return e;
    }
};

template <class R>
inline Phys<R> convert_phys(const Phys<double> &p) {
    Phys<R> o;
    o.omega_p = (R)p.omega_p;
    o.omega_m = (R)p.omega_m;
    o.A = (R)p.A;
    o.B = (R)p.B;
    o.ep_l = (R)p.ep_l;
    o.inv_l = (R)p.inv_l;
    for (int k = 0; k < 3; ++k) o.g[k] = (R)p.g[k];
    o.rho0 = (R)p.rho0;
    o.rho_ref = (R)p.rho_ref;
    o.scale = (R)p.scale;
    o.inv_scale = (R)p.inv_scale;
    o.flux_on = p.flux_on;
    o.src_on = p.src_on;
    o.ctu_on = p.ctu_on;
    o.divu_on = p.divu_on;
    o.gk = (R)p.gk;
    o.fene = p.fene;
    o.fene_L2 = (R)p.fene_L2;
    o.eta_p = (R)p.eta_p;
    o.lam = (R)p.lam;
    for (int c = 0; c < MAX_WALL; ++c)
        for (int k = 0; k < 3; ++k) o.wall_vel[c][k] = (R)p.wall_vel[c][k];
    return o;
}

template <class S>
struct Launch {
    using R = typename Store<S>::R;

    // split schedule: the stream-collide writes u[ucur] and the stress update reads it;
    // fused schedule: the stress update reads u[ucur], the stream-collide writes u[ucur^1].
    static KArgs<S> args(const DevState &d, bool fused = false) {
        KArgs<S> a;
        a.g = d.g;
        a.ph = convert_phys<R>(d.ph);
        a.f = (S *)d.f;
        a.tau = (const R *)d.tau[d.cur];
        a.tau_out = (R *)d.tau[d.cur ^ 1];
        a.u_in = (const R *)d.u[d.ucur];
        a.u_out = (R *)d.u[fused ? d.ucur ^ 1 : d.ucur];
        a.flag = d.flag;
        a.mask = d.mask;
        a.parts = d.parts;
        a.step = d.step;
        a.bad = d.bad;
        a.zlo = d.zlo;
        a.zhi = d.zhi > 0 ? d.zhi : d.g.nz;
        a.key_base = d.key_base;
        link_dirs<S>(a);
        return a;
    }
    // per-cell kernels: blocks of block_x x (128 / block_x) threads
    static dim3 block2(const DevState &d) { return dim3((unsigned)d.block_x, (unsigned)(128 / d.block_x)); }
    static int zcount(const DevState &d) { return (d.zhi > 0 ? d.zhi : d.g.nz) - d.zlo; }
    static dim3 grid2(const DevState &d) {
        const dim3 b = block2(d);
        return dim3((unsigned)((d.g.nx + b.x - 1) / b.x), (unsigned)((d.g.ny + b.y - 1) / b.y), (unsigned)zcount(d));
    }
    static dim3 grid3(const DevState &d) { return dim3((unsigned)((d.g.nx + d.block_x - 1) / d.block_x), d.g.ny, d.g.nz); }

    static cudaError_t init(const DevState &d, const double *rho, const double *u, const double *tau, long long r0,
                            long long count, long long ld, cudaStream_t s) {
        if (count <= 0) return cudaSuccess;
        KArgs<S> a = args(d);
        const unsigned nb = (unsigned)((count + 255) / 256);
        k_init<S><<<nb, 256, 0, s>>>(a, rho, u, tau, (R *)d.tau[d.cur], r0, count, ld);
        return cudaGetLastError();
    }
    // The row-pipelined stream-collide (k_lb_rows): rows of a multiple of 32 cells, at
    // most LR_MAX_NX, 16-byte aligned field arrays, a layout that fits the
    // shared memory of one block, Oldroyd-B or Giesekus stress (FENE-P reads conformation
    // tensors: per-cell kernel).  The result is bitwise that of the per-cell kernel.
    static size_t rows_smem(int nx) { return RowsLayout<S>{nx}.total(); }
    static bool rows_ok(const DevState &d) {
        auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
        if (d.ph.fene || d.g.nx % 32 != 0 || d.g.nx < 64 || d.g.nx > LR_MAX_NX) return false;
        // schedule AUTO: grids of 2^22 cells and more in the FP32 / 16-bit modes (measured
        // on GB300: at 128^3 the two stream-collides take the same time, below it the
        // per-cell kernel is faster, the row pipeline's per-block fill not being hidden;
        // the FP64 parity mode keeps the per-cell kernel)
        if (d.auto_kernels == 1 && (d.g.n < (1LL << 22) || !Store<S>::shifted)) return false;
        if (!al(d.f) || !al(d.tau[0]) || !al(d.tau[1]) || !al(d.mask) || !al(d.u[0]) || !al(d.u[1])) return false;
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return false;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
        return rows_smem(d.g.nx) <= (size_t)optin;
    }
    // rows per strip: enough strips for ~16 waves of resident blocks (d.lb_rows_yc > 0:
    // that many), at least 8 rows
    static RowsWork rows_work(const DevState &d, size_t smem) {
        const int ny = d.g.ny, nzc = zcount(d);
        int yc = d.lb_rows_yc;
        if (yc <= 0) {
            int dev = 0, sms = 148, smpb = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) {
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                cudaDeviceGetAttribute(&smpb, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            }
            long long per_sm = smpb > 0 ? (long long)smpb / (long long)(smem + 1024) : 1;
            if (per_sm < 1) per_sm = 1;
            const long long want = 16LL * sms * per_sm;
            long long strips = (want + nzc - 1) / nzc;
            if (strips < 1) strips = 1;
            yc = (int)((ny + strips - 1) / strips);
            if (yc < 8) yc = 8;
        }
        if (yc > ny) yc = ny;
        RowsWork w;
        w.yc = yc;
        w.strips = (ny + yc - 1) / yc;
        return w;
    }
    static cudaError_t lb_rows(const DevState &d, int parity, cudaStream_t s) {
        KArgs<S> a = args(d);
        const size_t sm = rows_smem(d.g.nx);
        const RowsWork w = rows_work(d, sm);
        static SmemAttrOnce attr[2];
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        // the attribute is the largest layout any nx up to LR_MAX_NX needs, within the limit
        const size_t lim = std::min(rows_smem(LR_MAX_NX), (size_t)optin);
        e = parity == 0 ? attr[0].ensure(k_lb_rows<S, 0>, lim) : attr[1].ensure(k_lb_rows<S, 1>, lim);
        if (e != cudaSuccess) return e;
        const unsigned nblk = (unsigned)(zcount(d) * w.strips);
        const unsigned nthr = (unsigned)(d.g.nx + 32);
        if (parity == 0)
            k_lb_rows<S, 0><<<nblk, nthr, sm, s>>>(a, w);
        else
            k_lb_rows<S, 1><<<nblk, nthr, sm, s>>>(a, w);
        return cudaGetLastError();
    }
    static int lb_rows_used(const DevState &d) { return d.auto_kernels && rows_ok(d) ? 1 : 0; }
    static cudaError_t lb(const DevState &d, int parity, cudaStream_t s) {
        if (d.auto_kernels && rows_ok(d)) return lb_rows(d, parity, s);
        KArgs<S> a = args(d);
        if (d.ph.fene) {  // the polymer force takes the stress of each cell's conformation
            if (parity == 0)
                k_lb<S, 0, true><<<grid2(d), block2(d), 0, s>>>(a);
            else
                k_lb<S, 1, true><<<grid2(d), block2(d), 0, s>>>(a);
        } else if (parity == 0) {
            k_lb<S, 0><<<grid2(d), block2(d), 0, s>>>(a);
        } else {
            k_lb<S, 1><<<grid2(d), block2(d), 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    // z-planes per block of the z-marching stress update (enough blocks for ~16 waves)
    static int fv_zchunk(const DevState &d) {
        const int nz = zcount(d);
        if (d.fv_zchunk > 0) return d.fv_zchunk < nz ? d.fv_zchunk : nz;
        const long long tiles = (long long)((d.g.nx + FV_X - 1) / FV_X) * ((d.g.ny + FV_Y - 1) / FV_Y);
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long want = 16LL * LBVE_FV_MIN_BLOCKS * sms;  // ~16 waves of resident blocks
        const long long chunks = (want + tiles - 1) / tiles;
        long long zc = (nz + chunks - 1) / chunks;
        if (zc < 16) zc = 16;
        if (zc > nz) zc = nz;
        return (int)zc;
    }
    // the VAR builds of the stress kernels: a finite-volume variant, FENE-P, or the flux or
    // the source switched off (the plain build has both on at compile time)
    static bool fv_variant(const DevState &d) {
        return d.ph.ctu_on || d.ph.divu_on || d.ph.gk != 0.0 || d.ph.fene || !d.ph.flux_on || !d.ph.src_on;
    }
    template <bool VAR, bool ZR, bool W16>
    static cudaError_t fv_launch(const DevState &d, unsigned nblk, int zc, cudaStream_t s) {
        KArgs<S> a = args(d);
        const size_t sm = sizeof(FvSmem<R, FvTile<FV_X, W16>::HN>);
        static SmemAttrOnce attr;
        cudaError_t e = attr.ensure(k_fv_tiled<S, VAR, ZR, W16>, sm);
        if (e != cudaSuccess) return e;
        k_fv_tiled<S, VAR, ZR, W16><<<nblk, FV_X * FV_Y, sm, s>>>(a, zc);
        return cudaGetLastError();
    }
    // planes staged by 16-byte copies: 4-byte reals, rows of whole 16-byte chunks and
    // 16-byte aligned stress and velocity arrays
    static bool fv_w16(const DevState &d) {
        auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
        return sizeof(R) == 4 && d.g.nx % 4 == 0 && al(d.tau[0]) && al(d.tau[1]) && al(d.u[0]) && al(d.u[1]);
    }
    template <bool VAR>
    static cudaError_t fv_var(const DevState &d, cudaStream_t s) {
        const int zc = fv_zchunk(d);
        const int tiles = ((d.g.nx + FV_X - 1) / FV_X) * ((d.g.ny + FV_Y - 1) / FV_Y);
        const unsigned nblk = (unsigned)(tiles * ((zcount(d) + zc - 1) / zc));
        const bool zr = d.zhi > 0;  // a z-slab: planes [zlo, zhi) only
        if constexpr (sizeof(R) == 4) {
            if (fv_w16(d)) return zr ? fv_launch<VAR, true, true>(d, nblk, zc, s) : fv_launch<VAR, false, true>(d, nblk, zc, s);
        }
        return zr ? fv_launch<VAR, true, false>(d, nblk, zc, s) : fv_launch<VAR, false, false>(d, nblk, zc, s);
    }
    // The two-cell stress kernel (k_fv_pair): schedule AUTO, the shifted modes' plain
    // build (flux and source on, no variant), nx a multiple of 4 (16-byte staging) and
    // 16-byte aligned stress, velocity and mask arrays.  Bitwise the tiled kernel's result.
    static bool fv_pair_ok(const DevState &d) {
        if constexpr (!Store<S>::shifted) {
            return false;
        } else {
            auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
            if (!d.auto_kernels || fv_variant(d) || d.g.nx % 4 != 0) return false;
            // schedule AUTO: grids of 2^21 cells and more (measured on GB300: 12 % faster at
            // 128^3, slower below about 10^6 cells, where its 512-cell columns leave SMs idle)
            if (d.auto_kernels == 1 && d.g.n < (1LL << 21)) return false;
            return al(d.tau[0]) && al(d.tau[1]) && al(d.u[0]) && al(d.u[1]) && al(d.mask);
        }
    }
    static int fv_pair_used(const DevState &d) { return fv_pair_ok(d) ? 1 : 0; }
    // z-planes per block of the two-cell stress kernel (~16 waves of 2 resident blocks)
    static int fv_pair_zchunk(const DevState &d) {
        const int nz = zcount(d);
        if (d.fv_zchunk > 0) return d.fv_zchunk < nz ? d.fv_zchunk : nz;
        const long long tiles = (long long)((d.g.nx + FP_TX - 1) / FP_TX) * ((d.g.ny + FP_TY - 1) / FP_TY);
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long want = 16LL * 2 * sms;
        const long long chunks = (want + tiles - 1) / tiles;
        long long zc = (nz + chunks - 1) / chunks;
        if (zc < 16) zc = 16;
        if (zc > nz) zc = nz;
        return (int)zc;
    }
    static cudaError_t fv_pair(const DevState &d, cudaStream_t s) {
        if constexpr (!Store<S>::shifted) {
            return cudaErrorInvalidValue;
        } else {
            KArgs<S> a = args(d);
            const int zc = fv_pair_zchunk(d);
            const int tiles = ((d.g.nx + FP_TX - 1) / FP_TX) * ((d.g.ny + FP_TY - 1) / FP_TY);
            const unsigned nblk = (unsigned)(tiles * ((zcount(d) + zc - 1) / zc));
            const size_t sm = sizeof(FvPairSmem);
            static SmemAttrOnce attr[2];
            const bool zr = d.zhi > 0;  // a z-slab: planes [zlo, zhi) only
            cudaError_t e = zr ? attr[1].ensure(k_fv_pair<S, true>, sm) : attr[0].ensure(k_fv_pair<S, false>, sm);
            if (e != cudaSuccess) return e;
            if (zr)
                k_fv_pair<S, true><<<nblk, FP_NT, sm, s>>>(a, zc);
            else
                k_fv_pair<S, false><<<nblk, FP_NT, sm, s>>>(a, zc);
            return cudaGetLastError();
        }
    }
    static cudaError_t fv(const DevState &d, cudaStream_t s) {
        if (fv_pair_ok(d)) return fv_pair(d, s);
        return fv_variant(d) ? fv_var<true>(d, s) : fv_var<false>(d, s);
    }
    static cudaError_t momentum_exchange(const DevState &d, int parity, const long long *links, const int *seg_begin,
                                         const int *seg_count, int nseg, int max_len, double *contrib, cudaStream_t s) {
        if (nseg <= 0 || max_len <= 0) return cudaSuccess;
        KArgs<S> a = args(d);
        const dim3 g((unsigned)((max_len + 127) / 128), (unsigned)nseg);
        if constexpr (Store<S>::shifted) {
            // reduced modes: per-block partials (nseg x ceil(max_len / 128) of them)
            if (parity == 0)
                k_momentum_exchange_part<S, 0><<<g, 128, 0, s>>>(a, links, seg_begin, seg_count, contrib);
            else
                k_momentum_exchange_part<S, 1><<<g, 128, 0, s>>>(a, links, seg_begin, seg_count, contrib);
        } else {
            // FP64 parity mode: one contribution per link, summed in link order
            if (parity == 0)
                k_momentum_exchange<S, 0><<<g, 128, 0, s>>>(a, links, seg_begin, seg_count, contrib);
            else
                k_momentum_exchange<S, 1><<<g, 128, 0, s>>>(a, links, seg_begin, seg_count, contrib);
        }
        return cudaGetLastError();
    }
    static cudaError_t halo_pack(const DevState &d, int what, int side, int parity, void *buf, cudaStream_t s) {
        KArgs<S> a = args(d);
        k_halo_pack<S><<<dim3((unsigned)((d.g.nx + 127) / 128), (unsigned)d.g.ny), 128, 0, s>>>(a, what, side, parity, buf);
        return cudaGetLastError();
    }
    static cudaError_t halo_unpack(const DevState &d, int what, int side, int parity, const void *buf,
                                   cudaStream_t s) {
        KArgs<S> a = args(d);
        k_halo_unpack<S><<<dim3((unsigned)((d.g.nx + 127) / 128), (unsigned)d.g.ny), 128, 0, s>>>(a, what, side, parity,
                                                                                                    buf);
        return cudaGetLastError();
    }
    static cudaError_t build_mask(const DevState &d, int lx, int ly, int lz, int ex, int ey, int ez, cudaStream_t s);
    static cudaError_t voxelise(const DevState &d, int p, const PartDev &host, cudaStream_t s) {
        KArgs<S> a = args(d);
        k_voxelise<S><<<64, 256, 0, s>>>(a, d.parts, p, d.flag, (R *)d.tau[0], (R *)d.tau[1]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const BBox b = particle_bbox(d.g, host.X, host.R, 3);
        return build_mask(d, b.lo[0], b.lo[1], b.lo[2], b.ext[0], b.ext[1], b.ext[2], s);
    }
    static cudaError_t particle_update(const DevState &d, int nparts, cudaStream_t s) {
        if (nparts <= 0) return cudaSuccess;
        k_particle_update<S><<<1, 64, 0, s>>>(d.parts, nparts);
        return cudaGetLastError();
    }
    static cudaError_t particle_links(const DevState &d, int nparts, long long *links, const int *seg_begin,
                                      int *seg_count, int first_seg, const int *capacity, cudaStream_t s) {
        if (nparts <= 0) return cudaSuccess;
        k_particle_links<S><<<nparts, 256, 0, s>>>(d.g, d.parts, d.flag, links, seg_begin, seg_count, first_seg,
                                                   capacity);
        return cudaGetLastError();
    }
    static cudaError_t fill_drain(const DevState &d, int parity, int nparts, uint8_t *kind, uint8_t *nf, double *delta,
                                  int *conv, double *diag, cudaStream_t s) {
        if (nparts <= 0) return cudaSuccess;
        KArgs<S> a = args(d);
        R *tau = (R *)d.tau[d.cur];
        if (parity == 0)
            k_fill_drain<S, 0><<<1, 512, 0, s>>>(a, d.parts, nparts, d.flag, d.mask, tau, kind, nf, delta, conv, diag);
        else
            k_fill_drain<S, 1><<<1, 512, 0, s>>>(a, d.parts, nparts, d.flag, d.mask, tau, kind, nf, delta, conv, diag);
        return cudaGetLastError();
    }
    static cudaError_t build_mask_impl(const DevState &d, int lx, int ly, int lz, int ex, int ey, int ez,
                                       cudaStream_t s) {
        const long long cells = (long long)ex * ey * ez;
        if (cells <= 0) return cudaSuccess;
        const unsigned nb = (unsigned)std::min<long long>((cells + 255) / 256, 65535);
        k_build_mask<S><<<nb, 256, 0, s>>>(d.g, d.flag, d.mask, lx, ly, lz, ex, ey, ez, (R *)d.tau[0], (R *)d.tau[1]);
        return cudaGetLastError();
    }
    static cudaError_t fused(const DevState &d, int parity, int zchunk, cudaStream_t s) {
        KArgs<S> a = args(d, true);
        FusedWork w;
        w.tiles_x = (d.g.nx + FT_X - 1) / FT_X;
        w.tiles_y = (d.g.ny + FT_Y - 1) / FT_Y;
        w.zchunk = zchunk;
        w.nzchunks = (d.g.nz + zchunk - 1) / zchunk;
        const size_t sm = sizeof(FusedSmem<R>);
        static SmemAttrOnce attr[2];
        cudaError_t e = parity == 0 ? attr[0].ensure(k_fused<S, 0>, sm) : attr[1].ensure(k_fused<S, 1>, sm);
        if (e != cudaSuccess) return e;
        const unsigned nblk = (unsigned)w.tiles_x * w.tiles_y * w.nzchunks;
        if (parity == 0)
            k_fused<S, 0><<<nblk, FT_X * FT_Y, sm, s>>>(a, w);
        else
            k_fused<S, 1><<<nblk, FT_X * FT_Y, sm, s>>>(a, w);
        return cudaGetLastError();
    }
    static cudaError_t read(const DevState &d, int parity, double *rho, double *u, double *tau, int z0, int z1,
                            long long ld, cudaStream_t s) {
        if (z1 <= z0) return cudaSuccess;
        KArgs<S> a = args(d);
        dim3 g = grid3(d);
        g.z = (unsigned)(z1 - z0);
        if (parity == 0)
            k_read<S, 0><<<g, d.block_x, 0, s>>>(a, rho, u, tau, z0, ld);
        else
            k_read<S, 1><<<g, d.block_x, 0, s>>>(a, rho, u, tau, z0, ld);
        return cudaGetLastError();
    }
    static cudaError_t pdfs_io(const DevState &d, int parity, double *io, int write, cudaStream_t s) {
        KArgs<S> a = args(d);
        if (parity == 0)
            k_pdfs_io<S, 0><<<grid3(d), d.block_x, 0, s>>>(a, io, write);
        else
            k_pdfs_io<S, 1><<<grid3(d), d.block_x, 0, s>>>(a, io, write);
        return cudaGetLastError();
    }
    static cudaError_t reduce(const DevState &d, int parity, double *partial, long long *nblocks, cudaStream_t s) {
        KArgs<S> a = args(d);
        dim3 g(grid3(d).x, d.g.ny, d.g.nz);
        // the reduction kernel needs exactly 256 threads per block
        g.x = (unsigned)((d.g.nx + 255) / 256);
        *nblocks = (long long)g.x * g.y * g.z;
        if (!partial) return cudaSuccess;
        if (parity == 0)
            k_reduce<S, 0><<<g, 256, 0, s>>>(a, partial);
        else
            k_reduce<S, 1><<<g, 256, 0, s>>>(a, partial);
        return cudaGetLastError();
    }

    static cudaError_t probe(const DevState &d, int parity, const long long *cells, int count, double *out,
                             cudaStream_t s) {
        if (count <= 0) return cudaSuccess;
        KArgs<S> a = args(d);
        const unsigned nb = (unsigned)((count + 127) / 128);
        if (parity == 0)
            k_probe<S, 0><<<nb, 128, 0, s>>>(a, cells, count, out);
        else
            k_probe<S, 1><<<nb, 128, 0, s>>>(a, cells, count, out);
        return cudaGetLastError();
    }

    // default tiles of a solve in the batched kernels (the pool autotuner may pick others)
    static int default_lb_tx(const DevState &) { return 32; }
    static int default_fv_tx(const DevState &) { return 32; }
    static void batch_tiles(const DevState &d, int lb_tx, int fv_tx, int *lb_eff, int *fv_eff) {
        *lb_eff = (lb_tx == 16 || lb_tx == 32 || lb_tx == 64 || lb_tx == 128) ? lb_tx : default_lb_tx(d);
        *fv_eff = FvBatchTiles<R>::ok(fv_tx) ? fv_tx : default_fv_tx(d);
    }
    static void fill_entry(const DevState &d, int parity, int lb_first, int fv_first, int fv_zchunk, int lb_tx,
                           int fv_tx, void *entry, int *lb_items, int *fv_items) {
        BatchEntry<S> &e = *reinterpret_cast<BatchEntry<S> *>(entry);
        e.a[0] = args(d);
        DevState d1 = d;  // odd steps of a launch sequence: stress ping-pong swapped
        d1.cur ^= 1;
        e.a[1] = args(d1);
        e.parity0 = parity;
        batch_tiles(d, lb_tx, fv_tx, &e.lb_tx, &e.fv_tx);
        const int lth = BLB_X * BLB_Y / e.lb_tx, fth = FV_NT / e.fv_tx;
        e.lb_first = lb_first;
        e.lb_items = ((d.g.nx + e.lb_tx - 1) / e.lb_tx) * ((d.g.ny + lth - 1) / lth) * d.g.nz;
        e.fv_first = fv_first;
        e.fv_zchunk = fv_zchunk > 0 ? fv_zchunk : fv_zchunk_of(d);
        e.fv_items = ((d.g.nx + e.fv_tx - 1) / e.fv_tx) * ((d.g.ny + fth - 1) / fth) *
                     ((d.g.nz + e.fv_zchunk - 1) / e.fv_zchunk);
        *lb_items = e.lb_items;
        *fv_items = e.fv_items;
    }
    static int fv_zchunk_of(const DevState &d) { return fv_zchunk(d); }
    static cudaError_t lb_batched(const void *entries, int n, int total, int k, int grid, const unsigned *dstep,
                                  int parity, cudaStream_t s) {
        if (total <= 0) return cudaSuccess;
        if (parity == 0)
            k_lb_batched<S, 0><<<grid, BLB_X * BLB_Y, 0, s>>>((const BatchEntry<S> *)entries, n, total, k, dstep);
        else
            k_lb_batched<S, 1><<<grid, BLB_X * BLB_Y, 0, s>>>((const BatchEntry<S> *)entries, n, total, k, dstep);
        return cudaGetLastError();
    }
    template <int TX, bool VAR>
    static cudaError_t fv_batched_tx(const void *entries, int n, int total, int k, int grid, cudaStream_t s) {
        const size_t sm = sizeof(FvSmem<R, FvTile<TX>::HN>);
        static SmemAttrOnce attr;
        cudaError_t e = attr.ensure(k_fv_batched<S, TX, VAR>, sm);
        if (e != cudaSuccess) return e;
        k_fv_batched<S, TX, VAR><<<grid, FV_NT, sm, s>>>((const BatchEntry<S> *)entries, n, total, k);
        return cudaGetLastError();
    }
    template <bool VAR>
    static cudaError_t fv_batched_var(const void *entries, int n, int total, int k, int grid, int tx, cudaStream_t s) {
        if constexpr (FvBatchTiles<R>::wide) {
            if (tx == 16) return fv_batched_tx<16, VAR>(entries, n, total, k, grid, s);
            if (tx == 64) return fv_batched_tx<64, VAR>(entries, n, total, k, grid, s);
        }
        return fv_batched_tx<32, VAR>(entries, n, total, k, grid, s);
    }
    static cudaError_t fv_batched(const void *entries, int n, int total, int k, int grid, int tx, int var,
                                  cudaStream_t s) {
        if (total <= 0) return cudaSuccess;
        return var ? fv_batched_var<true>(entries, n, total, k, grid, tx, s)
                   : fv_batched_var<false>(entries, n, total, k, grid, tx, s);
    }
    // resident blocks per SM of the batched stress kernel (both builds are held to the
    // same launch bound, so one grid serves both)
    template <int TX>
    static int fv_resident() {
        int per = 1;
        const size_t sm = sizeof(FvSmem<R, FvTile<TX>::HN>);
        cudaFuncSetAttribute(k_fv_batched<S, TX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fv_batched<S, TX, false>, FV_NT, sm);
        return per;
    }
    static int fv_variant_of(const DevState &d) { return fv_variant(d) ? 1 : 0; }
    // d: the member's state when the entries are built; step k after that uses the stress
    // ping-pong after the step's swap (cur ^ 1 for even k) and AA parity parity0 ^ (k & 1)
    static void fill_part_entry(const DevState &d, int parity0, const PartScratch &ps, void *entry) {
        PartEntry<S> &e = *reinterpret_cast<PartEntry<S> *>(entry);
        DevState d0 = d;
        d0.cur ^= 1;
        e.a[0] = args(d0);
        e.a[1] = args(d);
        e.parity0 = parity0;
        e.nparts = ps.nparts;
        e.first_seg = ps.first_seg;
        e.parts = d.parts;
        e.flag = d.flag;
        e.mask = d.mask;
        e.kind = ps.kind;
        e.nf = ps.nf;
        e.delta = ps.delta;
        e.diag = ps.diag;
        e.conv = ps.conv;
        e.links = ps.links;
        e.seg_begin = ps.seg_begin;
        e.seg_count = ps.seg_count;
        e.capacity = ps.capacity;
    }
    static cudaError_t particle_phase_batched(const void *entries, int n, int k, cudaStream_t s) {
        if (n <= 0) return cudaSuccess;
        k_particle_phase_batched<S><<<n, 512, 0, s>>>((const PartEntry<S> *)entries, k);
        return cudaGetLastError();
    }
    // resident blocks of the persistent grids: which = 0 for the stream-collide, else the
    // stress kernel of tile width `which`
    static int batched_grid(int which) {
        int dev = 0, sms = 148, per = 1;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (which == 0) {
            int per1 = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lb_batched<S, 0>, BLB_X * BLB_Y, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_lb_batched<S, 1>, BLB_X * BLB_Y, 0);
            per = std::min(per, per1);
        } else {
            per = fv_resident<32>();
            if constexpr (FvBatchTiles<R>::wide) {
                if (which == 16) per = fv_resident<16>();
                if (which == 64) per = fv_resident<64>();
            }
        }
        cudaGetLastError();
        if (per < 1) per = 1;
        return sms * per;
    }
    static cudaError_t residual(const DevState &d, void *usnap, double *partial, int nblocks, cudaStream_t s) {
        k_residual<S><<<nblocks, 256, 0, s>>>(d.g, d.mask, (const R *)d.u[d.ucur], (R *)usnap, partial);
        return cudaGetLastError();
    }

    static const KernelTable *table(int prec);
};

template <class S>
cudaError_t Launch<S>::build_mask(const DevState &d, int lx, int ly, int lz, int ex, int ey, int ez, cudaStream_t s) {
    return build_mask_impl(d, lx, ly, lz, ex, ey, ez, s);
}

template <class S>
const KernelTable *Launch<S>::table(int prec) {
        static const KernelTable t = {prec,           sizeof(S),        sizeof(R),   &init,
                                      &lb,            &fv,              &momentum_exchange, &voxelise,
                                      &particle_update, &particle_links, &fill_drain, &read,
                                      &pdfs_io,       &reduce,          &probe,      &build_mask,
                                      &fused,         sizeof(BatchEntry<S>), &fill_entry, &lb_batched,
                                      &fv_batched,    &batched_grid,    &residual,   &batch_tiles,
                                      &fv_zchunk_of,  &fv_variant_of,   sizeof(PartEntry<S>), &fill_part_entry,
                                      &particle_phase_batched, &halo_pack, &halo_unpack, &lb_rows_used, &fv_pair_used};
        return &t;
}

} // namespace lbve

// lbve_rows.cuh -- row-pipelined stream-collide (the LB half of one step of the coupled
// LB + Oldroyd-B method, Kuron et al., arXiv:2009.12279, Eqs. (lb), (guo), (force),
// (ubb)) for single solves whose x-rows fit in shared memory.
//
// A block owns one strip of consecutive x-rows of one plane and walks it in y.  One
// producer warp moves every operand of a row into a shared-memory ring with bulk
// asynchronous copies (the TMA engine, cp.async.bulk) that complete on mbarriers; the
// consumer threads, one per cell of the row, never wait on a global load:
//   * the 19 PDF rows the cells read: on an even step the row itself, on an odd step,
//     for direction i, row (y - c_iy, z - c_iz) of the array of -i, of which cell x
//     takes element x - c_ix (periodic wrap by index);
//   * the neighbour-mask row;
//   * the z-face stress components (xz, yz, zz) of rows (y, z - 1) and (y, z + 1);
//   * the stress rows y - 1, y, y + 1 of the plane, kept in a ring (each row is copied
//     once per strip and serves three consecutive rows).
// That is 32 copies per row, one per lane of the producer warp.
// A whole row holds every x neighbour, so the periodic wrap in x is an index and every
// copy is an aligned run of nx elements (nx a multiple of 32).  Rows are wrapped in y
// and z by their coordinates, exactly as the per-cell kernel wraps its neighbour
// indices, and every cell runs the per-cell kernel's arithmetic (lb_core_f): the results
// are bitwise those of k_lb.  Stores (post-collision PDFs, bounces, u) go straight to
// global memory; they do not stall the thread.
//
// Every wait is bounded: after LR_WAIT_NS nanoseconds a thread gives up, writes 2 to the
// status word (a.bad, when present) and leaves the strip; the producer, before it returns,
// waits (bounded again) until every copy it issued has landed.
#pragma once

#include "lbve_kernels.cuh"

namespace lbve {

// Stages of PDF / mask / z-face stress rows: as many as the shared memory of one block
// holds at nx = 512 (a stage holds the rows of one x-row of cells; every stage but the one
// being computed is in flight, which hides the DRAM latency)
template <class S>
__host__ __device__ constexpr int lr_stages() {
    return sizeof(S) == 2 ? 4 : (sizeof(S) == 4 ? 3 : 2);
}
// ring of in-plane stress rows: y - 1, y, y + 1 of the row computed, and the rows of the
// stages in flight
template <class S>
__host__ __device__ constexpr int lr_tring() {
    return lr_stages<S>() + 2;
}
constexpr int LR_MAX_NX = 512;             // one consumer thread per cell of a row
constexpr unsigned long long LR_WAIT_NS = 1000000000ull;  // 1 s

// ---------------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX ISA: mbarrier, cp.async.bulk)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity to complete; false after LR_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned k = 1;; ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 255u) == 0u && global_ns() - t0 > LR_WAIT_NS) return false;
    }
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to this block's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Shared-memory layout of the row pipeline for rows of nx cells.
template <class S>
struct RowsLayout {
    using R = typename Store<S>::R;
    int nx;
    __host__ __device__ size_t pdf_bytes() const { return (size_t)Q * nx * sizeof(S); }
    __host__ __device__ size_t mask_bytes() const { return (size_t)nx * 4; }
    __host__ __device__ size_t row6_bytes() const { return (size_t)6 * nx * sizeof(R); }
    __host__ __device__ size_t row3_bytes() const { return (size_t)3 * nx * sizeof(R); }
    __host__ __device__ size_t stage_bytes() const { return pdf_bytes() + mask_bytes() + 2 * row3_bytes(); }
    // barriers first (128 bytes), then the stages, then the stress ring
    __host__ __device__ size_t stage_off(int s) const { return 128 + (size_t)s * stage_bytes(); }
    __host__ __device__ size_t ring_off(int k) const {
        return 128 + (size_t)lr_stages<S>() * stage_bytes() + (size_t)k * row6_bytes();
    }
    __host__ __device__ size_t total() const { return ring_off(lr_tring<S>()); }
};

// Strip of rows: plane z, rows [y0, y0 + rows).
struct RowsWork {
    int strips;  // strips per plane
    int yc;      // rows per strip (the last one may be shorter)
};

__device__ __forceinline__ int wrap_coord(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// z-face stress components of the polymer force (Eq. (force) on the faces -+z reads
// tau_zj, j = x, y, z): xz, yz, zz, the staged order of the z-face rows
__host__ __device__ constexpr int zface_comp(int q) { return q == 0 ? 4 : (q == 1 ? 5 : 2); }
__host__ __device__ constexpr int zface_slot(int c) { return c == 4 ? 0 : (c == 5 ? 1 : 2); }

template <class S, int PAR>
__global__ void __launch_bounds__(LR_MAX_NX + 32, 1) k_lb_rows(KArgs<S> a, RowsWork w) {
    using R = typename Store<S>::R;
    constexpr int NS = lr_stages<S>(), T = lr_tring<S>();
    extern __shared__ __align__(128) unsigned char lr_smem[];
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const RowsLayout<S> L{nx};
    uint64_t *full = reinterpret_cast<uint64_t *>(lr_smem);
    uint64_t *empty = full + NS;
    const int nwarps_c = nx >> 5;  // consumer warps
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = a.zlo + blockIdx.x / w.strips;
    const int y0 = (blockIdx.x % w.strips) * w.yc;
    const int rows = min(w.yc, ny - y0);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (unsigned)nwarps_c);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned nxu = (unsigned)nx, nxy = (unsigned)nx * (unsigned)ny;
    auto row_of = [&](int y_, int z_) -> unsigned { return nxu * (unsigned)y_ + nxy * (unsigned)z_; };
    auto pdf_s = [&](int s, int i) -> S * { return reinterpret_cast<S *>(lr_smem + L.stage_off(s)) + (size_t)i * nx; };
    auto mask_s = [&](int s) -> uint32_t * {
        return reinterpret_cast<uint32_t *>(lr_smem + L.stage_off(s) + L.pdf_bytes());
    };
    // z-face stress rows of stage s: h 0 the -z row, 1 the +z row; q the z-face component
    auto tz_s = [&](int s, int h, int q) -> R * {
        return reinterpret_cast<R *>(lr_smem + L.stage_off(s) + L.pdf_bytes() + L.mask_bytes()) +
               ((size_t)h * 3 + q) * nx;
    };
    auto ring_s = [&](int k, int c) -> R * { return reinterpret_cast<R *>(lr_smem + L.ring_off(k)) + (size_t)c * nx; };
    const unsigned rowb_f = (unsigned)(nx * sizeof(S)), rowb_r = (unsigned)(nx * sizeof(R));

    if (warp == nwarps_c) {
        // ---------------- producer warp ----------------
        // row j of the strip (y = y0 + j) goes to stage j % NS; the in-plane stress row
        // y0 + k (k = -1 .. rows) to ring slot (k + 1) % T, so that row j reads ring slots
        // j, j + 1, j + 2 (mod T).  The slot refilled at row j held row y0 + j - NS - 1,
        // last read by row j - NS, whose stage the producer has seen released.
        const int zm = wrap_coord(z - 1, nz), zp = wrap_coord(z + 1, nz);
        bool ok = true;
        int issued = 0;
        for (int j = 0; j < rows && ok; ++j) {
            const int s = j % NS;
            if (j >= NS) ok = mbar_wait(&empty[s], (unsigned)((j / NS) - 1) & 1u);
            ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
            if (!ok) break;
            const int y = y0 + j;
            unsigned bytes = Q * rowb_f + (unsigned)nx * 4u + 12u * rowb_r;
            if (j == 0) bytes += 12u * rowb_r;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
            __syncwarp();
            // one copy per lane: lanes 0..18 the PDF rows, 19 the mask row, 20..25 the z-face
            // stress rows, 26..31 the in-plane stress row y + 1; at the strip's start lanes
            // 0..11 also copy the in-plane rows y0 - 1 and y0
            if (lane < Q) {
                const int i = lane;
                const S *src;
                if (PAR == 0) {
                    src = a.fq[i] + row_of(y, z);
                } else {
                    const int ys = wrap_coord(y - cy(i), ny), zs = wrap_coord(z - cz(i), nz);
                    src = a.fq[copp(i)] + row_of(ys, zs);
                }
                bulk_copy_g2s(pdf_s(s, i), src, rowb_f, &full[s]);
            } else if (lane == Q) {
                bulk_copy_g2s(mask_s(s), a.mask + row_of(y, z), (unsigned)nx * 4u, &full[s]);
            } else if (lane < 26) {
                const int h = (lane - 20) / 3, q = (lane - 20) % 3;
                bulk_copy_g2s(tz_s(s, h, q), a.tq[zface_comp(q)] + row_of(y, h == 0 ? zm : zp), rowb_r, &full[s]);
            } else {
                const int c = lane - 26, yn = wrap_coord(y + 1, ny);
                bulk_copy_g2s(ring_s((j + 2) % T, c), a.tq[c] + row_of(yn, z), rowb_r, &full[s]);
            }
            if (j == 0 && lane < 12) {
                const int k = lane / 6, c = lane % 6;  // k 0: row y0 - 1, 1: row y0
                const int yr = k == 0 ? wrap_coord(y0 - 1, ny) : y0;
                bulk_copy_g2s(ring_s(k, c), a.tq[c] + row_of(yr, z), rowb_r, &full[s]);
            }
            ++issued;
        }
        // every copy issued lands before the block exits: wait for the last stages' phases
        if (lane == 0) {
            for (int j = max(0, issued - NS); j < issued; ++j) {
                if (!mbar_wait(&full[j % NS], (unsigned)(j / NS) & 1u)) ok = false;
            }
            if (!ok && a.bad != nullptr) *(volatile unsigned *)a.bad = 2u;
        }
        return;
    }

    // ---------------- consumer threads: cell x of every row ----------------
    const int x = tid;
    for (int j = 0; j < rows; ++j) {
        const int s = j % NS;
        if (!mbar_wait(&full[s], (unsigned)(j / NS) & 1u)) {
            if (a.bad != nullptr) *(volatile unsigned *)a.bad = 2u;
            return;
        }
        const int y = y0 + j;
        const uint32_t m = mask_s(s)[x];
        if (!(m & 1u)) {
            const Cell cl(a.g, x, y, z);
            const unsigned r = cl.self();
            R f[Q], tr[6];
            const R inv = a.ph.inv_scale;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int xs = PAR == 0 ? x : (cx(i) == 0 ? x : (cx(i) > 0 ? cl.xm : cl.xp));
                f[i] = Store<S>::ld(pdf_s(s, i) + xs, inv);
            }
            const int km = j % T, kc = (j + 1) % T, kp = (j + 2) % T;
#pragma unroll
            for (int c = 0; c < 6; ++c) tr[c] = ring_s(kc, c)[x];
            auto tn = [&](int l, int c) -> R {
                switch (l) {
                    case 0: return ring_s(kc, c)[cl.xp];
                    case 1: return ring_s(kc, c)[cl.xm];
                    case 2: return ring_s(kp, c)[x];
                    case 3: return ring_s(km, c)[x];
                    case 4: return tz_s(s, 1, zface_slot(c))[x];
                    default: return tz_s(s, 0, zface_slot(c))[x];
                }
            };
            lb_core_f<S, PAR>(a, cl, r, m, tr, tn, f);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

}  // namespace lbve

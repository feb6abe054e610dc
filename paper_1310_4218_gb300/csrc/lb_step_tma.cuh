// Persistent step kernel for FP32 split columns of one exact length NZ whose
// work items stream their input through shared memory with TMA: every warp
// owns one box slot, and as soon as its current item's box is in registers
// it starts the tensor copy of its next item's box, which then lands while
// the current item runs its k_c solves.
//
// Why.  A work item reads its 8x2 columns and their upwind neighbours, all
// NZ levels, before any arithmetic can start, and then runs its k_c solves
// (the serial-in-k recurrence of Fig. 1 / Fig. 4) without touching memory.
// With plain loads the next item's reads only start after the solves, and
// the loads in flight are bounded by the registers of the warps that happen
// to be in their load phase.  A tensor copy needs no registers and overlaps
// the whole solve phase.  Measured on GB300 this kernel is slower than the
// register-load kernels on every workload tried: the memory phase itself
// (not its overlap with the solves) bounds the step, and the slots leave
// room for only 16 warps at nz = 96.  It is an option
// (lb_options.staged_loads), not a default.
//
// Box.  An item's input is the 9x3 column neighbourhood of its 8x2 tile
// (upwind side on each axis, Sec. VI-B stencil).  TMA wants the innermost
// box coordinate on a 16-byte boundary, so the box is 12 x 3 x NZ floats
// starting at x rounded down to a multiple of 4; it covers every column the
// tile reads for either upwind direction.  Tiles whose neighbours wrap
// around the periodic x or y boundary are not boxed: the warp reads them
// from global memory as the register-load kernel does.
//
// Slot protocol.  Slot w belongs to warp w alone: one mbarrier, armed by
// lane 0 with the box's byte count right before the copy; the warp waits on
// it, reads the box, and only then issues the next copy into the same slot,
// so the barrier's phases alternate strictly with the warp's items and a
// parity wait is never ambiguous.  Waits give up after the kernel's time
// limit with LB_ETIMEOUT; copies in flight land before the CTA exits.
#pragma once

#include "lb_step_kernel.cuh"

namespace lbk {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait until the phase of the given parity has completed.  Gives up (false)
// after timeout_ns, or when *abort (may be null) is set by another warp of
// the CTA.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          long long timeout_ns, const volatile int *abort) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    unsigned it = 0;
    while (!mbar_test(bar, parity)) {
        if ((++it & 63u) == 0u) {
            if (abort && *abort) return false;
            if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
        }
    }
    return true;
}
// 3D tiled TMA load of one box into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_box(void *dst, const void *tmap, unsigned long long *bar,
                                             int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// ------------------------------------------------------------ box geometry
// Box origin of a tile at (x, y): one upwind column / row outside the tile
// on the upwind side, x rounded down to a multiple of 4 (16 bytes).
__device__ __forceinline__ int box_x0(const GridDev &g, int x) { return (x - (g.sx > 0 ? 1 : 0)) & ~3; }
__device__ __forceinline__ int box_y0(const GridDev &g, int y) { return y - (g.sy > 0 ? 1 : 0); }
// 1: some column of the tile reads a neighbour across the periodic boundary.
__device__ __forceinline__ int tile_wraps(const GridDev &g, int x, int y) {
    const bool wx = g.sx > 0 ? x == 0 : x + kTileW >= g.nx;
    const bool wy = g.sy > 0 ? y == 0 : y + kTileH >= g.ny;
    return (wx || wy) ? 1 : 0;
}

// A split item whose input box is in shared memory (box[(z * 3 + y) * 12 + x]
// relative to the box origin).  On return from the load phase (the
// advected column is in registers, every lane has read the box) `loaded()`
// runs: it reuses the slot for the next item.
template <int NZ, class Loaded>
__device__ __forceinline__ int process_item_box(const StepParams<float> &p, const GridDev &g,
                                                const VPDev &vp, int chunk, long long t, int src,
                                                int lane, bool do_mass, LaneSum<float> &acc,
                                                const float *box, const Loaded &loaded) {
    constexpr int H = NZ / 2;
    constexpr int kZ = kBoxW * kBoxH;          // floats per box level
    const SplitGeom sg = split_geom<NZ>(g, vp, chunk, lane);
    const int top = sg.top;
    const int kc = split_kc<NZ>(g, sg, t);
    const int xs = box_x0(g, sg.tx0), ys = box_y0(g, sg.ty0);
    const int bx = sg.i - xs, by = sg.j - ys;
    const int bc = by * kBoxW + bx;                      // the column
    const int ba = bc - g.sx;                            // upwind in x
    const int bb = bc - g.sy * kBoxW;                    // upwind in y
    const float *lev = box + (top ? (NZ - 1) * kZ : 0);  // local level 0 of this lane
    const int zst = top ? -kZ : kZ;

    float2 y2[H / 2];
    float *y = reinterpret_cast<float *>(y2);
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int m = 0; m < H / 2; ++m) {
            const float *l0 = lev + (2 * m) * zst, *l1 = l0 + zst;
            const float2 a = f2(l0[ba], l1[ba]);
            const float2 b = f2(l0[bb], l1[bb]);
            y2[m] = fma2(wy2, b, mul2(wx2, a));
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? NZ - 1 : 0;
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int k = top ? NZ - 1 - s : s;
            const float *l = lev + s * zst;
            float v = fmaT(wy, l[bb], wx * l[ba]);
            v = fmaT(k == kdown ? w0 + wz : w0, l[bc], v);
            const int ku = k - sz;
            if (ku >= 0 && ku < NZ) v = fmaT(wz, box[ku * kZ + bc], v);
            y[s] = v;
        }
    }
    __syncwarp();
    loaded();
    return split_finish<float, float, NZ>(p, g, sg, y2, kc, src, do_mass, acc);
}

// ------------------------------------------------------------ the kernel
// A popped work item, resolved far enough to start its box copy.
struct NextItem {
    int c;          // item index, -1: none left this step
    int boxed;      // 1: a box copy was issued for it
};

// Resolve item c and, unless its tile wraps, start the copy of its box into
// `slot` (lane 0 issues; the barrier is armed with the box's byte count).
template <int NZ>
__device__ __forceinline__ NextItem start_item(const StepParams<float> &p, int c, int src, int lane,
                                               float *slot, unsigned long long *bar) {
    NextItem nx{c, 0};
    if (c < 0) return nx;
    const int2 it = p.items[c];
    const VPDev vp = p.vps[it.x];
    const GridDev &g = p.grids[vp.grid];
    const int tiles_x = (vp.w + kTileW - 1) / kTileW;
    const int ty = it.y / tiles_x, tx = it.y - ty * tiles_x;
    const int x = vp.x0 + tx * kTileW, y = vp.y0 + ty * kTileH;
    if (tile_wraps(g, x, y)) return nx;
    nx.boxed = 1;
    if (lane == 0) {
        const void *map = static_cast<const char *>(p.tmaps) + (size_t)(2 * vp.grid + src) * 128;
        // this warp's reads of the slot (generic proxy) come before the
        // copy's writes (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, (unsigned)(kBoxW * kBoxH * NZ * 4));
        tma_load_box(slot, map, bar, box_x0(g, x), box_y0(g, y), 0);
    }
    return nx;
}

template <int NZ, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
lb_step_kernel_tma(const __grid_constant__ StepParams<float> p) {
    static_assert(NZ % 4 == 0 && NZ <= 256, "box depth");
    constexpr int kWarps = THREADS / kWarp;
    constexpr int kSlotFloats = kBoxW * kBoxH * NZ;
    static_assert((kSlotFloats * 4) % 128 == 0, "slots stay 128-byte aligned");
    extern __shared__ __align__(128) unsigned char s_dyn[];
    __shared__ unsigned long long s_bar[kWarps];
    __shared__ int s_ctr;
    __shared__ int s_flag;
    __shared__ unsigned long long s_t0, s_tend;

    const int bin = blockIdx.x;
    const int warp = threadIdx.x / kWarp;
    const int lane = threadIdx.x % kWarp;
    // slots: 128-byte aligned start inside the dynamic buffer, then the
    // per-warp sums
    const unsigned pad = (128u - (smem_addr(s_dyn) & 127u)) & 127u;
    float *slot = reinterpret_cast<float *>(s_dyn + pad) + (size_t)warp * kSlotFloats;
    double *s_mass = reinterpret_cast<double *>(s_dyn + pad + (size_t)kWarps * kSlotFloats * 4);
    unsigned long long *bar = &s_bar[warp];

    if (threadIdx.x == 0) {
        p.bin_smid[bin] = smid();
        p.bin_cal[4 * bin + 0] = (long long)globaltimer_ns();
        p.bin_cal[4 * bin + 1] = clock64();
        for (int n = 0; n < kWarps; ++n) mbar_init(&s_bar[n], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int ibeg = p.queue_mode ? 0 : p.bin_start[bin];
    const int iend = p.queue_mode ? p.nitems : p.bin_start[bin + 1];
    const long long t0 = p.dclock ? p.dclock[0] : p.t0;
    const int parity0 = p.dclock ? (int)p.dclock[1] : p.parity0;
    unsigned phase = 0;                            // parity of the slot's next copy
    int pending = 0;                               // 1: a copy into the slot is in flight
    unsigned long long wsweeps = 0;                // lane 0: cell-sweep updates
    bool failed = false;                           // CTA-uniform

    for (int s = 0; s < p.nsteps; ++s) {
        const long long t = t0 + s;
        const int src = (parity0 + s) & 1;
        const bool do_mass = p.mass_every > 0 && ((t + 1) % p.mass_every) == 0;

        if (bin == 0 && s > 0) reduce_mass<float, THREADS>(p, t0, s - 1);

        if (threadIdx.x == 0) {
            s_ctr = 0;
            s_tend = 0ull;
            s_t0 = (unsigned long long)clock64();
            if (bin == 0) p.qhead[(s + 1) & 1] = 0u;
            if (p.steal) p.bin_ctr[(size_t)((s + 1) & 1) * p.nbins + bin] = 0u;
        }
        if (do_mass)
            for (int n = threadIdx.x; n < kWarps * p.ngrids; n += THREADS) s_mass[n] = 0.0;
        __syncthreads();
        // the previous step's stores (generic proxy, any SM) are visible
        // after the grid barrier; order them before this step's copies
        asm volatile("fence.proxy.async.global;" ::: "memory");

        LaneSum<float> acc;
        int cur_grid = -1;
        NextItem cur = start_item<NZ>(p, pop_item(p, s, bin, lane, &s_ctr, ibeg, iend), src, lane,
                                      slot, bar);
        pending = cur.boxed;
        bool ok = true;
        while (cur.c >= 0) {
            const long long c0 = clock64();
            const int2 it = p.items[cur.c];
            const VPDev vp = p.vps[it.x];
            const GridDev &g = p.grids[vp.grid];
            if (do_mass && vp.grid != cur_grid) {
                if (cur_grid >= 0) {
                    double v = acc.take();
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) s_mass[warp * p.ngrids + cur_grid] += v;
                }
                cur_grid = vp.grid;
            }
            NextItem nxt{-1, 0};
            // once the current item's input is in registers: pop the next
            // item and start its copy, which lands during the solves
            auto loaded = [&]() {
                nxt = start_item<NZ>(p, pop_item(p, s, bin, lane, &s_ctr, ibeg, iend), src, lane,
                                     slot, bar);
            };
            int kc;
            if (cur.boxed) {
                if (!mbar_wait(bar, phase, p.timeout_ns, nullptr)) {
                    ok = false;
                    break;
                }
                phase ^= 1u;
                pending = 0;
                kc = process_item_box<NZ>(p, g, vp, it.y, t, src, lane, do_mass, acc, slot, loaded);
            } else {
                loaded();
                kc = process_item_split<float, float, NZ>(p, g, vp, it.y, t, src, lane, do_mass,
                                                          acc);
            }
            pending = nxt.boxed;
            __syncwarp();
            const long long c1 = clock64();
            const unsigned ksum = __reduce_add_sync(0xffffffffu, (unsigned)kc);
            if (lane == 0) {
                atomicAdd(&p.vp_cycles[it.x], (unsigned long long)(c1 - c0));
                wsweeps += (unsigned long long)ksum * (unsigned)g.nz;
            }
            cur = nxt;
        }
        if (!ok && lane == 0) atomicCAS(p.status, 0, (int32_t)LB_ETIMEOUT);
        if (do_mass && cur_grid >= 0) {
            double v = acc.take();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_mass[warp * p.ngrids + cur_grid] += v;
        }
        if (lane == 0) atomicMax(&s_tend, (unsigned long long)clock64());
        __syncthreads();
        if (threadIdx.x == 0 && s_tend > s_t0) p.bin_busy[bin] += s_tend - s_t0;
        if (do_mass) {
            for (int gi = threadIdx.x; gi < p.ngrids; gi += THREADS) {
                double v = 0.0;
                for (int w = 0; w < kWarps; ++w) v += s_mass[w * p.ngrids + gi];
                p.bin_mass[((size_t)(s & 1) * p.nbins + bin) * p.ngrids + gi] = v;
            }
        }
        if (!grid_barrier(p.bar, gridDim.x, p.timeout_ns, p.status, &s_flag)) {
            failed = true;
            break;
        }
    }

    if (lane == 0 && p.sweeps && wsweeps) atomicAdd(p.sweeps, wsweeps);
    // a copy still in flight (only after a failed wait) lands before the
    // CTA exits
    if (pending && lane == 0) mbar_wait(bar, phase, p.timeout_ns, nullptr);
    if (failed) return;
    if (bin == 0 && p.nsteps > 0) {
        reduce_mass<float, THREADS>(p, t0, p.nsteps - 1);
        if (p.dclock && threadIdx.x == 0) {
            p.dclock[0] = t0 + p.nsteps;
            p.dclock[1] = (parity0 + p.nsteps) & 1;
        }
    }
    if (threadIdx.x == 0) {
        p.bin_cal[4 * bin + 2] = (long long)globaltimer_ns();
        p.bin_cal[4 * bin + 3] = clock64();
    }
}

template <int NZ, int THREADS>
inline KernelInfo kernel_entry_tma() {
    KernelInfo k = kernel_entry<float, float, NZ, true, 1, THREADS, true>();
    k.fn = (const void *)&lb_step_kernel_tma<NZ, THREADS>;
    k.tma_slots = THREADS / kWarp;
    k.tma_slot_bytes = kBoxW * kBoxH * NZ * 4;
    return k;
}

}  // namespace lbk

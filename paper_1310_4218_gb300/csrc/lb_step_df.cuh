// Dataflow variant of the persistent step kernel: a launch's time steps
// without a grid barrier (lb_options.dataflow, atomic-queue mode).
//
// Why.  With a grid barrier every SM idles at the end of each step until
// the last work item of the step, anywhere on the GPU, has finished (the
// `barrier` stalls of the step kernel's profile).  Here the work items of
// all the launch's steps come from one queue (index step * nitems + item,
// the queue order within each step), and a warp starts item c at step s as
// soon as every item owning a column of c's closed 4-neighbourhood (c
// included) has finished step s - 1:
//   - read after write: every column c's step reads (its own and its four
//     neighbours, whatever the upwind side or the dynamics) holds step s's
//     input;
//   - write after read: every item that read c's columns at step s - 1 has
//     finished, so c may overwrite them in the ping-pong buffer.
// The arithmetic of every column is the barrier kernel's (run_item), so
// the fields are the same bit for bit.
//
// Bookkeeping per step (kDfSlots slots, reused every kDfSlots steps): a
// warp adds its finished-item count and its global-sum partials into the
// slot of its current step when it moves on to a later step or runs out
// of items; the flush that completes a step reduces it -- after the step
// before has been reduced, so the sums enter the history in step order --
// clears the slot and advances `reduced`.  A warp starts an item of step
// s >= kDfSlots only once step s - kDfSlots is reduced.  The reduction of
// the launch's last step advances the device clock once every CTA has
// read it.
//
// Ordering: a finished item publishes done[c] = s + 1 with a release (every
// lane fences after its stores, then lane 0 writes the flag) at the start of
// the warp's next iteration, after the next pop and table loads and before
// any wait (so no warp waits while holding an unpublished flag); waiting
// lanes read the flags with acquire loads, and a warp barrier orders every
// lane's loads of the item after them.  An item's dependency list (at most
// kDfDeps entries, else the CSR) and its table entries load before the
// waits, so the flags cost one load latency beside the table lookups.  Every wait is bounded by the ctx's time limit
// (LB_ETIMEOUT; a status set elsewhere ends the wait at once), after which
// the warp leaves the launch.  The protocol, with its deadlock freedom, is
// modelled on the host in tests/test_dataflow_model.py.
#pragma once

#include "lb_step_kernel.cuh"

namespace lbk {

__device__ __forceinline__ int df_ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Spin until *p >= want (true), or until the time limit or a status set
// elsewhere (false; the time limit records LB_ETIMEOUT).
__device__ __forceinline__ bool df_wait_ge(const int *p, int want, long long timeout_ns,
                                           int32_t *status) {
    if (df_ld_acquire(p) >= want) return true;
    const unsigned long long t0 = globaltimer_ns();
    unsigned it = 0;
    for (;;) {
        __nanosleep(64);
        if (df_ld_acquire(p) >= want) return true;
        if ((++it & 15u) == 0u) {
            if (*(volatile int32_t *)status != 0) return false;
            if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
                atomicCAS(status, 0, (int32_t)LB_ETIMEOUT);
                return false;
            }
        }
    }
}

// The warp's global-sum partial of one grid into step s's slot.
template <class TC>
__device__ __forceinline__ void df_add_mass(const StepParams<TC> &p, int s, int grid,
                                            LaneSum<TC> &acc, int lane) {
    double v = acc.take();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(&p.df_mass[(size_t)(s % kDfSlots) * p.ngrids + grid], v);
}

// Hand the warp's count (and sums) of step s to its slot; the flush that
// completes the step reduces it.  Warp-uniform; false after a failed wait.
template <class TC>
__device__ __forceinline__ bool df_flush(const StepParams<TC> &p, long long t0, int parity0,
                                         int s, int &cur_grid, unsigned &cnt, LaneSum<TC> &acc,
                                         int lane) {
    if (s < 0 || cnt == 0) return true;
    const long long t = t0 + s;
    const bool do_mass = p.mass_every > 0 && ((t + 1) % p.mass_every) == 0;
    if (do_mass && cur_grid >= 0) df_add_mass(p, s, cur_grid, acc, lane);
    cur_grid = -1;
    const int slot = s % kDfSlots;
    unsigned prev = 0;
    if (lane == 0) {
        __threadfence();                        // the sums before the count
        prev = atomicAdd(&p.df->cnt[slot], cnt);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    const bool last = prev + cnt == (unsigned)p.nitems;
    cnt = 0;
    if (!last) return true;
    int ok = 1;
    if (lane == 0) {
        __threadfence();
        ok = df_wait_ge(reinterpret_cast<const int *>(&p.df->reduced), s, p.timeout_ns, p.status);
        if (ok && do_mass) {
            const unsigned long long seq = *p.mass_seq;
            for (int gi = 0; gi < p.ngrids; ++gi) {
                double *m = &p.df_mass[(size_t)slot * p.ngrids + gi];
                const double sum = *(volatile double *)m;
                double *e = p.mass_hist + ((size_t)(seq % kMassHist) * p.ngrids + gi) * 2;
                e[0] = sum;
                e[1] = 0.0;
                if (!isfinite(sum)) atomicCAS(p.status, 0, (int32_t)LB_ENUMERIC);
                *m = 0.0;
            }
            p.mass_t[seq % kMassHist] = t;
            __threadfence();
            *p.mass_seq = seq + 1;
        }
        if (ok) {
            p.df->cnt[slot] = 0;
            if (s == p.nsteps - 1 && p.dclock) {
                ok = df_wait_ge(reinterpret_cast<const int *>(&p.df->started), (int)gridDim.x,
                                p.timeout_ns, p.status);
                if (ok) {
                    p.dclock[0] = t0 + p.nsteps;
                    p.dclock[1] = (parity0 + p.nsteps) & 1;
                }
            }
            __threadfence();
            atomicExch(&p.df->reduced, (unsigned)(s + 1));
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <class TS, class TC, int NZ, bool EXACT, int NZLO, int THREADS, bool TWIN>
__global__ void __launch_bounds__(THREADS, 1)
lb_step_kernel_df(const __grid_constant__ StepParams<TC> p) {
    __shared__ unsigned long long s_t0, s_tend;
    const int bin = blockIdx.x;
    const int lane = threadIdx.x % kWarp;

    if (threadIdx.x == 0) {
        p.bin_smid[bin] = smid();
        p.bin_cal[4 * bin + 0] = (long long)globaltimer_ns();
        p.bin_cal[4 * bin + 1] = clock64();
        s_t0 = (unsigned long long)clock64();
        s_tend = 0ull;
    }
    const long long t0 = p.dclock ? p.dclock[0] : p.t0;
    const int parity0 = p.dclock ? (int)p.dclock[1] : p.parity0;
    __syncthreads();                            // the whole CTA has read the clock
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&p.df->started, 1u);
    }

    const unsigned n = (unsigned)p.nitems;
    const unsigned long long total = (unsigned long long)p.nsteps * n;
    int cur_s = -1, cur_grid = -1;
    unsigned cnt = 0;
    LaneSum<TC> acc;
    bool ok = true;
    // the warp's last finished item, whose flag is published at the start
    // of the next iteration -- after the pop and the table loads, so that
    // the fence finds the item's stores drained -- and before any wait
    int pend = -1, pend_s = 0;
    auto publish = [&]() {
        if (pend >= 0) {
            __threadfence();                    // every lane's stores before the flag
            __syncwarp();
            if (lane == 0) atomicExch(p.df_done + pend, pend_s + 1);
            pend = -1;
        }
    };
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(&p.df->qhead, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= total) break;
        const int s = (int)(i / n), c = (int)(i % n);
        // the item's tables (never written during a launch) load beside its
        // dependency list, before the waits
        const int2 it = p.items[c];
        const int dl = (p.df_inl && lane < kDfDeps) ? p.df_inl[(size_t)c * kDfDeps + lane] : -1;
        const VPDev vp = p.vps[it.x];
        publish();
        if (s != cur_s) {
            if (!df_flush(p, t0, parity0, cur_s, cur_grid, cnt, acc, lane)) { ok = false; break; }
            cur_s = s;
        }
        // the slot of step s is free once step s - kDfSlots is reduced
        int w = 1;
        if (s >= kDfSlots && lane == 0)
            w = df_wait_ge(reinterpret_cast<const int *>(&p.df->reduced), s - kDfSlots + 1,
                           p.timeout_ns, p.status);
        if (!__shfl_sync(0xffffffffu, w, 0)) { ok = false; break; }
        // every item owning a column of c's closed neighbourhood has finished step s - 1
        if (s > 0) {
            bool got = true;
            if (p.df_inl) {
                if (dl >= 0) got = df_wait_ge(p.df_done + dl, s, p.timeout_ns, p.status);
            } else {
                for (int k = p.df_dep_start[c] + lane; k < p.df_dep_start[c + 1]; k += kWarp)
                    got = got && df_wait_ge(p.df_done + p.df_deps[k], s, p.timeout_ns, p.status);
            }
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            __syncwarp();                       // every lane's loads after the acquiring lanes'
        }

        const long long t = t0 + s;
        const int src = (parity0 + s) & 1;
        const bool do_mass = p.mass_every > 0 && ((t + 1) % p.mass_every) == 0;
        const GridDev &g = p.grids[vp.grid];
        if (do_mass && vp.grid != cur_grid) {
            if (cur_grid >= 0) df_add_mass(p, s, cur_grid, acc, lane);
            cur_grid = vp.grid;
        }
        const long long c0 = clock64();
        int kc;
        if (g.jacobi) {
            const ItemResult<TC> r = run_item_jacobi<TS, TC, NZ, EXACT, NZLO, false, TWIN>(
                p, &g, vp, it.y, t, src, lane, do_mass, acc);
            kc = r.kc;
            acc = r.acc;
        } else {
            kc = run_item<TS, TC, NZ, EXACT, NZLO, false, TWIN, false>(p, g, vp, it.y, t, src, lane,
                                                                       do_mass, acc);
        }
        __syncwarp();
        const long long c1 = clock64();
        const unsigned ksum = __reduce_add_sync(0xffffffffu, (unsigned)kc);
        if (lane == 0) {
            atomicAdd(&p.vp_cycles[it.x], (unsigned long long)(c1 - c0));
            if (p.sweeps) atomicAdd(p.sweeps, (unsigned long long)ksum * (unsigned)g.nz);
        }
        pend = c;
        pend_s = s;
        ++cnt;
    }
    if (ok) {
        publish();
        df_flush(p, t0, parity0, cur_s, cur_grid, cnt, acc, lane);
    }
    if (lane == 0) atomicMax(&s_tend, (unsigned long long)clock64());
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_tend > s_t0) p.bin_busy[bin] += s_tend - s_t0;
        p.bin_cal[4 * bin + 2] = (long long)globaltimer_ns();
        p.bin_cal[4 * bin + 3] = clock64();
    }
}

// The barrier kernel's entry with its dataflow variant attached.
template <int NZ, int THREADS>
inline KernelInfo kernel_entry_twin_df() {
    KernelInfo k = kernel_entry<float, float, NZ, true, 1, THREADS, false, 0, true>();
    k.df_fn = (const void *)&lb_step_kernel_df<float, float, NZ, true, 1, THREADS, true>;
    return k;
}

}  // namespace lbk

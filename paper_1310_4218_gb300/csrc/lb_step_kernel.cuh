// Persistent step kernel: every VP of every grid, nsteps time steps, one
// cooperative launch, one CTA (a "processor") per SM by default.
//
// Work decomposition.  A VP (Sec. III over-decomposition) is cut into work
// items: 8 x 2 column tiles (split kernels on half-warps), 16 x 2 tiles
// (split kernels on paired warps) or runs of 32 consecutive columns of its
// row-major column order (one lane per column: twin halves and plain
// Thomas).  A processor owns a contiguous range of the item table, and its
// warps pop items from a shared-memory counter, or with stealing from a
// per-processor global counter that idle processors also draw on.  In queue
// mode every warp pops from one global counter instead (the task-queue
// scheme of Sec. II).
//
// Per column and step (Fig. 2's dynamics then physics kernels, fused):
//   1. dynamics into registers, level by level and coalesced across the
//      warp (lanes are x-adjacent columns): upwind advection, or with
//      GridDev::jacobi one weighted 7-point Jacobi sweep (Sec. IV), run in
//      out-of-line copies of the item code;
//   2. k_c(i,j,t) from the moving-disk rule or the k_c array (Sec. VI-B);
//   3. k_c implicit vertical-diffusion solves in registers (the serial-in-k
//      recurrence of Fig. 1 / Fig. 4).  Split and twin forms use the
//      twisted factorisation: both halves of the column eliminate toward
//      the middle with the same pivots, solve a 2 x 2 middle system and
//      back-substitute outward.  The halves sit on two half-warps, on two
//      warps, or as packed FP32x2 pairs in one lane; FP64 and BF16 storage
//      use one lane per column with plain Thomas.  The column is shifted by
//      a reference value c before the solves and shifted back after:
//      M 1 = 1, so M^-k (d - c1) + c1 = M^-k d exactly, while the rounding
//      of the FP32 pivots acts on the small deviation d - c1 instead of d;
//   4. store of the new column; compensated sum of the stored values for
//      the global sum diagnostic.
// Each work item's duration (clock64) is added to its VP's cost: the
// on-device load measurement of Sec. V.  A grid-wide barrier with a time
// limit separates steps.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace lbk {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int smid() {
    int s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// ------------------------------------------------------------ storage I/O
template <class TS, class TC> struct IO;
template <> struct IO<float, float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ float st(float *p, float x) { *p = x; return x; }
};
template <> struct IO<double, double> {
    static __device__ __forceinline__ double ld(const double *p) { return *p; }
    static __device__ __forceinline__ double st(double *p, double x) { *p = x; return x; }
};
template <> struct IO<double, float> {
    static __device__ __forceinline__ float ld(const double *p) { return (float)*p; }
    static __device__ __forceinline__ float st(double *p, float x) { *p = (double)x; return x; }
};
template <> struct IO<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float st(__nv_bfloat16 *p, float x) {
        __nv_bfloat16 b = __float2bfloat16_rn(x);
        *p = b;
        return __bfloat162float(b);
    }
};

// ------------------------------------------------------------ compensated sums
// Per-lane accumulator of stored values.  FP32 compute: per column, the
// running sum and the exact rounding error of every addition (TwoSum, Knuth)
// are kept apart ("Sum2" of Ogita, Rump and Oishi, accurate as if summed in
// twice the working precision); the column's (sum, error) pair then goes
// into a double-float lane total, converted to FP64 only when flushed.
// FP64 compute: plain FP64 sums.
template <class TC> struct LaneSum;
template <> struct LaneSum<float> {
    float hi = 0.f, lo = 0.f;   // lane total
    float s = 0.f, e = 0.f;     // current column: sum, summed errors
    __device__ __forceinline__ void col_begin() { s = 0.f; e = 0.f; }
    __device__ __forceinline__ void add(float v) {
        float t = __fadd_rn(s, v);
        float bp = __fsub_rn(t, s);
        float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
        e = __fadd_rn(e, err);
        s = t;
    }
    __device__ __forceinline__ void col_end() {
        float t = __fadd_rn(hi, s);
        float bp = __fsub_rn(t, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(s, bp));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double take() {
        double v = (double)hi + (double)lo;
        hi = lo = 0.f;
        return v;
    }
};
template <> struct LaneSum<double> {
    double tot = 0.0, s = 0.0;
    __device__ __forceinline__ void col_begin() { s = 0.0; }
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ void col_end() { tot += s; }
    __device__ __forceinline__ double take() {
        double v = tot;
        tot = 0.0;
        return v;
    }
};

// ------------------------------------------------------------ load rule
// Moving disk (Sec. VI-B): k_in inside radius R of (x0,y0)+t(vx,vy), periodic
// minimum-image distance, exact integer arithmetic.
__device__ __forceinline__ int kc_disk(const GridDev &g, int i, int j, long long t) {
    long long cx = ((long long)g.disk_x0 + t * g.disk_vx) % g.nx;
    long long cy = ((long long)g.disk_y0 + t * g.disk_vy) % g.ny;
    if (cx < 0) cx += g.nx;
    if (cy < 0) cy += g.ny;
    int dx = i - (int)cx;
    int dy = j - (int)cy;
    if (dx < 0) dx += g.nx;
    if (dy < 0) dy += g.ny;
    if (dx > g.nx / 2) dx -= g.nx;
    if (dy > g.ny / 2) dy -= g.ny;
    long long d2 = (long long)dx * dx + (long long)dy * dy;
    return d2 <= (long long)g.disk_r * g.disk_r ? g.k_in : g.k_out;
}

// k_c of column (i, j) at step t: the disk rule, or the array entry (dense
// [ny][nx], whatever the field's row pitch) bounded to 0..LB_KC_MAX; an
// entry above the bound also sets the grid's range flag (every writer
// stores 1, so the race between lanes is harmless).
__device__ __forceinline__ int kc_at(const GridDev &g, int i, int j, int, long long t) {
    if (g.kc_disk) return kc_disk(g, i, j, t);
    int k = g.kc[j * g.nx + i];
    if (k > LB_KC_MAX) {
        k = LB_KC_MAX;
        *(volatile int32_t *)g.kc_range = 1;
    }
    return k > 0 ? k : 0;
}

template <class TC> __device__ __forceinline__ TC wgt(const GridDev &g, int n);
template <> __device__ __forceinline__ float wgt<float>(const GridDev &g, int n) { return g.wf[n]; }
template <> __device__ __forceinline__ double wgt<double>(const GridDev &g, int n) { return g.wd[n]; }
template <class TC> __device__ __forceinline__ TC mlast(const GridDev &g);
template <> __device__ __forceinline__ float mlast<float>(const GridDev &g) { return g.mlast_f; }
template <> __device__ __forceinline__ double mlast<double>(const GridDev &g) { return g.mlast_d; }
template <class TC> __device__ __forceinline__ TC rlast(const GridDev &g);
template <> __device__ __forceinline__ float rlast<float>(const GridDev &g) { return g.rlast_f; }
template <> __device__ __forceinline__ double rlast<double>(const GridDev &g) { return g.rlast_d; }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------------ Jacobi sweep
// The Sec. IV dynamics phase in its Jacobi form (GridDev.jacobi): one
// weighted Jacobi sweep of the 7-point stencil per step,
//     q*_k = (1 - 6 nu) q_k + nu (x-1, x+1, y-1, y+1 neighbours + q_{k-1} + q_{k+1}),
// periodic in x/y; at the vertical ends the missing neighbour is the cell
// itself (zero flux).  Plane offsets of a column's four lateral neighbours:
struct JacNbr {
    int oc, oxm, oxp, oym, oyp;
};
__device__ __forceinline__ JacNbr jac_nbr(const GridDev &g, int i, int j) {
    const int im = i > 0 ? i - 1 : g.nx - 1, ip = i + 1 < g.nx ? i + 1 : 0;
    const int jm = j > 0 ? j - 1 : g.ny - 1, jp = j + 1 < g.ny ? j + 1 : 0;
    return JacNbr{j * g.pitch + i, j * g.pitch + im, j * g.pitch + ip, jm * g.pitch + i,
                  jp * g.pitch + i};
}
template <class TC> __device__ __forceinline__ TC jac_nu(const GridDev &g);
template <> __device__ __forceinline__ float jac_nu<float>(const GridDev &g) { return g.nu_f; }
template <> __device__ __forceinline__ double jac_nu<double>(const GridDev &g) { return g.nu_d; }
template <class TC> __device__ __forceinline__ TC jac_w0(const GridDev &g);
template <> __device__ __forceinline__ float jac_w0<float>(const GridDev &g) { return g.w0j_f; }
template <> __device__ __forceinline__ double jac_w0<double>(const GridDev &g) { return g.w0j_d; }

// New value of level k (0 <= k < nz) of the column.
template <class TS, class TC>
__device__ __forceinline__ TC jacobi_level(const GridDev &g, const TS *in, int k, int nz,
                                           const JacNbr &n) {
    const int plane = g.plane, o = k * plane;
    const int kd = k > 0 ? k - 1 : 0, ku = k < nz - 1 ? k + 1 : nz - 1;
    TC s = IO<TS, TC>::ld(in + (o + n.oxm));
    s += IO<TS, TC>::ld(in + (o + n.oxp));
    s += IO<TS, TC>::ld(in + (o + n.oym));
    s += IO<TS, TC>::ld(in + (o + n.oyp));
    s += IO<TS, TC>::ld(in + (kd * plane + n.oc));
    s += IO<TS, TC>::ld(in + (ku * plane + n.oc));
    return fmaT(jac_nu<TC>(g), s, jac_w0<TC>(g) * IO<TS, TC>::ld(in + (o + n.oc)));
}

// ------------------------------------------------------------ one Thomas solve
// In place on y[0..nz-1]: forward p_k = (y_k + r p_{k-1}) m_k, back
// x_k = p_k + r m_k x_{k+1}.  EXACT: nz == NZ, every coefficient is a
// kernel-parameter constant.  Otherwise nz <= NZ at run time (warp-uniform):
// rows below nz-1 use the nz-independent table, row nz-1 the grid's
// last-row pivot (ml, rl = r*ml), and the forward sweep stops there.  Rows
// >= nz hold exact zeros that the forward sweep never touches, so the full
// back substitution leaves them zero and starts row nz-1 from x_nz = 0.
template <class TC, int NZ, bool EXACT, int NZLO>
__device__ __forceinline__ void thomas_solve(TC (&y)[NZ], const Coef<TC> &cf, int nz,
                                             TC ml, TC rl) {
    if (EXACT || NZLO > 1 || nz > 1) {
        TC p = y[0] * cf.m[0];
        y[0] = p;
#pragma unroll
        for (int k = 1; k < NZ; ++k) {
            if (EXACT || k < NZLO - 1 || k < nz - 1) {
                p = fmaT(p, cf.rm[k], y[k] * cf.m[k]);
                y[k] = p;
            } else if (k == nz - 1) {
                y[k] = fmaT(p, rl, y[k] * ml);
            }
        }
    } else {
        y[0] = y[0] * ml;
    }
#pragma unroll
    for (int k = NZ - 2; k >= 0; --k) y[k] = fmaT(cf.rm[k], y[k + 1], y[k]);
}

// ------------------------------------------------------------ one work item
// Column geometry of a lane within a work item.
struct ColGeom {
    int i, j, oc, oi, oj;
    bool active;
};

__device__ __forceinline__ ColGeom col_geom(const GridDev &g, const VPDev &vp, int chunk, int lane) {
    ColGeom c;
    const int q = chunk * kWarp + lane;
    c.active = q < vp.ncols;
    const int qq = c.active ? q : vp.ncols - 1;
    const int ly = qq / vp.w;
    c.i = vp.x0 + (qq - ly * vp.w);
    c.j = vp.y0 + ly;
    int im = c.i - g.sx, jm = c.j - g.sy;
    im = im < 0 ? im + g.nx : (im >= g.nx ? im - g.nx : im);
    jm = jm < 0 ? jm + g.ny : (jm >= g.ny ? jm - g.ny : jm);
    c.oc = c.j * g.pitch + c.i;
    c.oi = c.j * g.pitch + im;
    c.oj = jm * g.pitch + c.i;
    return c;
}

// Advection and the k_c solves: leaves the new column in y, minus cref.
template <class TS, class TC, int NZ, bool EXACT, int NZLO, bool JAC = false>
__device__ __forceinline__ int column_physics(const StepParams<TC> &p, const GridDev &g,
                                              const ColGeom &cg, long long t, int src,
                                              TC (&y)[NZ], TC &cref) {
    const int nz = EXACT ? NZ : g.nz;
    const TS *in = static_cast<const TS *>(g.q[src]);
    const int plane = g.plane;
    int kc = kc_at(g, cg.i, cg.j, cg.oc, t);
    if (!cg.active || !g.sweeps_on) kc = 0;

    // 1. advection (or the Jacobi sweep) into registers (rows >= nz: exact zeros)
    const TC wx = wgt<TC>(g, 1), wy = wgt<TC>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, cg.i, cg.j);
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            if (EXACT || k < NZLO || k < nz) y[k] = jacobi_level<TS, TC>(g, in, k, nz, jn);
            else y[k] = TC(0);
        }
    } else if (g.xy_only) {
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            if (EXACT || k < NZLO || k < nz) {
                TC a = IO<TS, TC>::ld(in + (k * plane + cg.oi));
                TC b = IO<TS, TC>::ld(in + (k * plane + cg.oj));
                y[k] = fmaT(wy, b, wx * a);
            } else {
                y[k] = TC(0);
            }
        }
    } else {
        // general form: own value, and the vertical upwind neighbour with
        // closed end faces (the cell at the closed downwind face keeps its
        // outflow, the cell at the closed upwind face gets no inflow)
        const TC w0 = wgt<TC>(g, 0), wz = wgt<TC>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? nz - 1 : 0;
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            if (EXACT || k < NZLO || k < nz) {
                TC c = IO<TS, TC>::ld(in + (k * plane + cg.oc));
                TC a = IO<TS, TC>::ld(in + (k * plane + cg.oi));
                TC b = IO<TS, TC>::ld(in + (k * plane + cg.oj));
                TC v = fmaT(wy, b, wx * a);
                v = fmaT(k == kdown ? w0 + wz : w0, c, v);
                const int ku = k - sz;
                if (ku >= 0 && ku < nz) v = fmaT(wz, IO<TS, TC>::ld(in + (ku * plane + cg.oc)), v);
                y[k] = v;
            } else {
                y[k] = TC(0);
            }
        }
    }

    // 2.-3. shift, k_c implicit solves (the shift back happens at the store)
    cref = TC(0);
    if (kc > 0) {
        cref = y[EXACT ? NZ / 2 : 0];
#pragma unroll
        for (int k = 0; k < NZ; ++k)
            if (EXACT || k < NZLO || k < nz) y[k] -= cref;
        const TC ml = EXACT ? TC(0) : mlast<TC>(g);
        const TC rl = EXACT ? TC(0) : rlast<TC>(g);
        for (int s = 0; s < kc; ++s) thomas_solve<TC, NZ, EXACT, NZLO>(y, p.coef, nz, ml, rl);
    }
    return kc;
}

// 4. shift back, store, compensated sum of the stored values.
template <class TS, class TC, int NZ, bool EXACT, int NZLO, bool MASS>
__device__ __forceinline__ void store_column(const GridDev &g, const ColGeom &cg, int src,
                                             const TC (&y)[NZ], TC cref, LaneSum<TC> &acc) {
    const int nz = EXACT ? NZ : g.nz;
    TS *out = static_cast<TS *>(g.q[src ^ 1]);
    const int plane = g.plane;
    if (!cg.active) return;
    if (MASS) acc.col_begin();
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
        if (EXACT || k < NZLO || k < nz) {
            TC xs = IO<TS, TC>::st(out + (k * plane + cg.oc), y[k] + cref);
            if (MASS) acc.add(xs);
        }
    }
    if (MASS) acc.col_end();
}

// Returns the lane's k_c (0 for lanes past the VP's last column).
template <class TS, class TC, int NZ, bool EXACT, int NZLO, bool JAC = false>
__device__ __forceinline__ int process_item(const StepParams<TC> &p, const GridDev &g,
                                            const VPDev &vp, int chunk, long long t, int src,
                                            int lane, bool do_mass, LaneSum<TC> &acc) {
    const ColGeom cg = col_geom(g, vp, chunk, lane);
    TC y[NZ];
    TC cref;
    const int kc = column_physics<TS, TC, NZ, EXACT, NZLO, JAC>(p, g, cg, t, src, y, cref);
    if (do_mass) store_column<TS, TC, NZ, EXACT, NZLO, true>(g, cg, src, y, cref, acc);
    else store_column<TS, TC, NZ, EXACT, NZLO, false>(g, cg, src, y, cref, acc);
    return kc;
}

// ------------------------------------------------------------ split columns
// Two lanes per column: lane l (l < 16) holds levels 0..H-1 of the item's
// column l, lane l+16 holds levels NZ-1..H of the same column, both indexed
// by the distance s from their own end (H = NZ/2).  A solve is the twisted
// ("burn at both ends") factorisation of the tridiagonal system: both lanes
// eliminate toward the middle at once -- M is symmetric under k -> NZ-1-k,
// so both use the same pivots m_s of a column that starts at a zero-flux
// end -- then exchange their last eliminated values p (own) and p' (other,
// one shuffle) and solve the 2x2 middle system
//     x_own = (p + a p') / (1 - a^2),   a = r m_{H-1},
// and back-substitute outward.  Same operation count as one lane running
// the whole column, half the registers per thread and half the dependence
// chain per solve.
// Packed FP32 pairs (sm_100+ f32x2 instructions) for independent work on two
// levels: advection, shift, and two interleaved compensated sums.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Sum2 (TwoSum errors kept apart) on two interleaved chains at once.
struct PairSum {
    float2 s, e;
    __device__ __forceinline__ void begin() {
        s = f2(0.f, 0.f);
        e = f2(0.f, 0.f);
    }
    __device__ __forceinline__ void add(float2 v) {
        const float2 m1 = f2(-1.f, -1.f);
        const float2 t = add2(s, v);
        const float2 bp = fma2(s, m1, t);       // t - s
        const float2 a1 = fma2(bp, m1, t);      // t - bp
        const float2 a2 = fma2(a1, m1, s);      // s - (t - bp)
        const float2 a3 = fma2(bp, m1, v);      // v - bp
        e = add2(e, add2(a2, a3));
        s = t;
    }
};

// Lane geometry within an 8x2 tile: item = kTileW x kTileH tile of the VP,
// tiles in row-major order; lane pair (c, c + 16) holds column c of the tile.
struct SplitGeom {
    int top;              // 1: upper half of the column
    int i, j;             // column (clamped to the VP for inactive lanes)
    int tx0, ty0;         // tile origin in grid coordinates
    int oc, oi, oj;       // plane offsets of the column and its upwind neighbours
    int lbase, lstep;     // element offset of local level s: lbase + s * lstep
    bool active;
};

template <int NZ>
__device__ __forceinline__ SplitGeom split_geom(const GridDev &g, const VPDev &vp, int chunk,
                                                int lane) {
    constexpr int kCols = kWarp / 2;
    static_assert(kTileW * kTileH == kCols, "a tile is one column per lane pair");
    SplitGeom sg;
    sg.top = lane >> 4;
    const int c = lane & (kCols - 1);
    const int tiles_x = (vp.w + kTileW - 1) / kTileW;
    const int ty = chunk / tiles_x, tx = chunk - ty * tiles_x;
    const int xi = tx * kTileW + (c % kTileW), yi = ty * kTileH + c / kTileW;
    sg.active = xi < vp.w && yi < vp.h;
    sg.tx0 = vp.x0 + tx * kTileW;
    sg.ty0 = vp.y0 + ty * kTileH;
    sg.i = vp.x0 + (xi < vp.w ? xi : vp.w - 1);
    sg.j = vp.y0 + (yi < vp.h ? yi : vp.h - 1);
    int im = sg.i - g.sx, jm = sg.j - g.sy;
    im = im < 0 ? im + g.nx : (im >= g.nx ? im - g.nx : im);
    jm = jm < 0 ? jm + g.ny : (jm >= g.ny ? jm - g.ny : jm);
    sg.oc = sg.j * g.pitch + sg.i;
    sg.oi = sg.j * g.pitch + im;
    sg.oj = jm * g.pitch + sg.i;
    sg.lbase = sg.top ? (NZ - 1) * g.plane : 0;
    sg.lstep = sg.top ? -g.plane : g.plane;
    return sg;
}

template <int NZ>
__device__ __forceinline__ int split_kc(const GridDev &g, const SplitGeom &sg, long long t) {
    int kc = kc_at(g, sg.i, sg.j, sg.oc, t);
    if (!sg.active || !g.sweeps_on) kc = 0;
    return kc;
}

// Shift, k_c twisted solves, shift back, store and compensated sum: the part
// of a split item after its advected column is in y2 (levels 2m, 2m+1 of the
// lane's half in y2[m]).  Returns the column's k_c on the lower lane, 0 on
// the upper one.
template <class TS, class TC, int NZ>
__device__ __forceinline__ int split_finish(const StepParams<TC> &p, const GridDev &g,
                                            const SplitGeom &sg, float2 (&y2)[NZ / 4], int kc,
                                            int src, bool do_mass, LaneSum<TC> &acc) {
    constexpr int H = NZ / 2;
    constexpr int kCols = kWarp / 2;
    const int top = sg.top;
    float *y = reinterpret_cast<float *>(y2);
    TS *out = static_cast<TS *>(g.q[src ^ 1]);

    // shift by the column's level H-1 value (held by the bottom lane)
    const float mid = __shfl_xor_sync(0xffffffffu, y[H - 1], kCols);
    const float cref = kc > 0 ? (top ? mid : y[H - 1]) : 0.f;
    if (kc > 0) {
        const float2 nc = f2(-cref, -cref);
#pragma unroll
        for (int m = 0; m < H / 2; ++m) y2[m] = add2(y2[m], nc);
    }
    const Coef<TC> &cf = p.coef;
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)kc);
    int rc = cf.resc_every;
    for (int r = 0; r < kmax; ++r) {
        const bool act = r < kc;
        if (act) {
            float pp = y[0] * cf.e[0];
            y[0] = pp;
#pragma unroll
            for (int s = 1; s < H; ++s) {
                pp = fmaT(pp, cf.rm[s], y[s] * cf.e[s]);
                y[s] = pp;
            }
        }
        const float other = __shfl_xor_sync(0xffffffffu, y[H - 1], kCols);
        if (act) {
            y[H - 1] = fmaT(cf.ifa, other, y[H - 1]) * cf.ifc;
#pragma unroll
            for (int s = H - 2; s >= 0; --s) y[s] = fmaT(cf.rm[s], y[s + 1], y[s]);
            if (--rc == 0) {
                rc = cf.resc_every;
                const float2 rs = f2(cf.resc, cf.resc);
#pragma unroll
                for (int m = 0; m < H / 2; ++m) y2[m] = mul2(y2[m], rs);
            }
        }
    }

    if (sg.active) {
        const float2 c2 = f2(cref, cref), fk2 = f2(cf.f[kc], cf.f[kc]);
        PairSum ps;
        if (do_mass) ps.begin();
#pragma unroll
        for (int m = 0; m < H / 2; ++m) {
            const float2 x = fma2(fk2, y2[m], c2);
            out[sg.lbase + (2 * m) * sg.lstep + sg.oc] = x.x;
            out[sg.lbase + (2 * m + 1) * sg.lstep + sg.oc] = x.y;
            if (do_mass) ps.add(x);
        }
        if (do_mass) {
            // fold the two chains into the lane's column sum
            acc.col_begin();
            acc.s = ps.s.x;
            acc.e = ps.e.x;
            acc.add(ps.s.y);
            acc.e = __fadd_rn(acc.e, ps.e.y);
            acc.col_end();
        }
    }
    return top ? 0 : kc;
}

template <class TS, class TC, int NZ, bool JAC = false>
__device__ __forceinline__ int process_item_split(const StepParams<TC> &p, const GridDev &g,
                                                  const VPDev &vp, int chunk, long long t,
                                                  int src, int lane, bool do_mass,
                                                  LaneSum<TC> &acc) {
    static_assert(sizeof(TS) == 4 && sizeof(TC) == 4, "split kernels are FP32");
    constexpr int H = NZ / 2;
    static_assert(H % 2 == 0, "levels are processed in pairs");
    const SplitGeom sg = split_geom<NZ>(g, vp, chunk, lane);
    const int top = sg.top, lbase = sg.lbase, lstep = sg.lstep;
    const int oc = sg.oc, oi = sg.oi, oj = sg.oj;
    const int plane = g.plane;
    const TS *in = static_cast<const TS *>(g.q[src]);
    const int kc = split_kc<NZ>(g, sg, t);

    float2 y2[H / 2];                  // levels 2m, 2m+1 in one register pair
    float *y = reinterpret_cast<float *>(y2);
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, sg.i, sg.j);
#pragma unroll
        for (int s = 0; s < H; ++s) y[s] = jacobi_level<TS, TC>(g, in, top ? NZ - 1 - s : s, NZ, jn);
    } else if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int m = 0; m < H / 2; ++m) {
            const int off0 = lbase + (2 * m) * lstep, off1 = off0 + lstep;
            const float2 a = f2(IO<TS, TC>::ld(in + (off0 + oi)), IO<TS, TC>::ld(in + (off1 + oi)));
            const float2 b = f2(IO<TS, TC>::ld(in + (off0 + oj)), IO<TS, TC>::ld(in + (off1 + oj)));
            y2[m] = fma2(wy2, b, mul2(wx2, a));
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? NZ - 1 : 0;
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int k = top ? NZ - 1 - s : s;
            const int off = lbase + s * lstep;
            float c = IO<TS, TC>::ld(in + (off + oc));
            float a = IO<TS, TC>::ld(in + (off + oi));
            float b = IO<TS, TC>::ld(in + (off + oj));
            float v = fmaT(wy, b, wx * a);
            v = fmaT(k == kdown ? w0 + wz : w0, c, v);
            const int ku = k - sz;
            if (ku >= 0 && ku < NZ) v = fmaT(wz, IO<TS, TC>::ld(in + (ku * plane + oc)), v);
            y[s] = v;
        }
    }
    return split_finish<TS, TC, NZ>(p, g, sg, y2, kc, src, do_mass, acc);
}

// Split columns for grids of any nz in [2, 2 * HMAX] (several grids of
// different nz in one launch): the lower lane holds the ceil(nz/2) lowest
// levels, the upper lane the floor(nz/2) highest, each counted from its own
// end.  Both eliminate toward the middle with the same nz-independent
// pivots of a column that starts at a zero-flux end; the middle 2x2 system
// couples them with the grid's a_b, a_t.  The lane's half length is a
// runtime value, so no per-level branch may depend on it (the compiler
// could turn it into a loop bound and move the column out of registers):
// loads read a clamped level, selects keep levels beyond the half at zero,
// and stores are predicated in PTX.
__device__ __forceinline__ void st_pred(float *ptr, float v, bool pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}"
                 :: "l"(ptr), "f"(v), "r"((unsigned)pred) : "memory");
}

template <class TS, class TC, int HMAX, bool JAC = false>
__device__ __forceinline__ int process_item_split_rt(const StepParams<TC> &p, const GridDev &g,
                                                     const VPDev &vp, int chunk, long long t,
                                                     int src, int lane, bool do_mass,
                                                     LaneSum<TC> &acc) {
    static_assert(sizeof(TS) == 4 && sizeof(TC) == 4, "split kernels are FP32");
    static_assert(HMAX % 2 == 0, "levels are processed in pairs");
    constexpr int kCols = kWarp / 2;
    static_assert(kTileW * kTileH == kCols, "a tile is one column per lane pair");
    const int top = lane >> 4;
    const int c = lane & (kCols - 1);
    const int tiles_x = (vp.w + kTileW - 1) / kTileW;
    const int ty = chunk / tiles_x, tx = chunk - ty * tiles_x;
    const int xi = tx * kTileW + (c % kTileW), yi = ty * kTileH + c / kTileW;
    const bool active = xi < vp.w && yi < vp.h;
    const int i = vp.x0 + (xi < vp.w ? xi : vp.w - 1);
    const int j = vp.y0 + (yi < vp.h ? yi : vp.h - 1);
    int im = i - g.sx, jm = j - g.sy;
    im = im < 0 ? im + g.nx : (im >= g.nx ? im - g.nx : im);
    jm = jm < 0 ? jm + g.ny : (jm >= g.ny ? jm - g.ny : jm);
    const int plane = g.plane, nz = g.nz;
    const int hlen = top ? nz / 2 : (nz + 1) / 2;     // levels this lane holds
    const int oc = j * g.pitch + i, oi = j * g.pitch + im, oj = jm * g.pitch + i;
    const int lbase = top ? (nz - 1) * plane : 0;
    const int lstep = top ? -plane : plane;
    const TS *in = static_cast<const TS *>(g.q[src]);
    TS *out = static_cast<TS *>(g.q[src ^ 1]);

    int kc = kc_at(g, i, j, oc, t);
    if (!active || !g.sweeps_on) kc = 0;

    float2 y2[HMAX / 2];
    float *y = reinterpret_cast<float *>(y2);
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, i, j);
#pragma unroll
        for (int s = 0; s < HMAX; ++s) {
            const int sc = min(s, hlen - 1);
            const float v = jacobi_level<TS, TC>(g, in, top ? nz - 1 - sc : sc, nz, jn);
            y[s] = s < hlen ? v : 0.f;
        }
    } else if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int m = 0; m < HMAX / 2; ++m) {
            const int s0 = min(2 * m, hlen - 1), s1 = min(2 * m + 1, hlen - 1);
            const int off0 = lbase + s0 * lstep, off1 = lbase + s1 * lstep;
            const float2 a = f2(IO<TS, TC>::ld(in + (off0 + oi)), IO<TS, TC>::ld(in + (off1 + oi)));
            const float2 b = f2(IO<TS, TC>::ld(in + (off0 + oj)), IO<TS, TC>::ld(in + (off1 + oj)));
            const float2 v = fma2(wy2, b, mul2(wx2, a));
            y2[m] = f2(2 * m < hlen ? v.x : 0.f, 2 * m + 1 < hlen ? v.y : 0.f);
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? nz - 1 : 0;
#pragma unroll
        for (int s = 0; s < HMAX; ++s) {
            const int sc = min(s, hlen - 1);
            const int k = top ? nz - 1 - sc : sc;
            const int off = lbase + sc * lstep;
            const float cc = IO<TS, TC>::ld(in + (off + oc));
            const float a = IO<TS, TC>::ld(in + (off + oi));
            const float b = IO<TS, TC>::ld(in + (off + oj));
            float v = fmaT(wy, b, wx * a);
            v = fmaT(k == kdown ? w0 + wz : w0, cc, v);
            const int ku = k - sz;
            const int kuc = ku < 0 ? 0 : (ku >= nz ? nz - 1 : ku);
            const float u = IO<TS, TC>::ld(in + (kuc * plane + oc));
            v = (ku >= 0 && ku < nz) ? fmaT(wz, u, v) : v;
            y[s] = s < hlen ? v : 0.f;
        }
    }

    // shift by the column's level ceil(nz/2)-1 value (the lower lane's last)
    float last = 0.f;
#pragma unroll
    for (int s = 0; s < HMAX; ++s) last = s == hlen - 1 ? y[s] : last;
    const float mid = __shfl_xor_sync(0xffffffffu, last, kCols);
    const float cref = kc > 0 ? (top ? mid : last) : 0.f;
    if (kc > 0) {
        const float2 nc = f2(-cref, -cref);
#pragma unroll
        for (int m = 0; m < HMAX / 2; ++m) y2[m] = add2(y2[m], nc);
    }
    const Coef<TC> &cf = p.coef;
    const float ifa = top ? g.ifa_t_f : g.ifa_b_f, ifc = g.ifc_bt_f;
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)kc);
    int rc = cf.resc_every;
    for (int r = 0; r < kmax; ++r) {
        const bool act = r < kc;
        float pp = 0.f;
        if (act) {
            pp = y[0] * cf.e[0];
            y[0] = pp;
#pragma unroll
            for (int s = 1; s < HMAX; ++s) {
                const float np = fmaT(pp, cf.rm[s], y[s] * cf.e[s]);
                const bool in_half = s < hlen;
                y[s] = in_half ? np : y[s];
                pp = in_half ? np : pp;
            }
        }
        const float other = __shfl_xor_sync(0xffffffffu, pp, kCols);
        if (act) {
            const float xl = fmaT(ifa, other, pp) * ifc;
            y[HMAX - 1] = hlen == HMAX ? xl : y[HMAX - 1];
#pragma unroll
            for (int s = HMAX - 2; s >= 0; --s) {
                const float bk = fmaT(cf.rm[s], y[s + 1], y[s]);
                y[s] = s == hlen - 1 ? xl : (s < hlen - 1 ? bk : y[s]);
            }
            if (--rc == 0) {
                rc = cf.resc_every;
                const float2 rs = f2(cf.resc, cf.resc);
#pragma unroll
                for (int m = 0; m < HMAX / 2; ++m) y2[m] = mul2(y2[m], rs);
            }
        }
    }

    const float2 c2 = f2(cref, cref), fk2 = f2(cf.f[kc], cf.f[kc]);
    PairSum ps;
    if (do_mass) ps.begin();
#pragma unroll
    for (int m = 0; m < HMAX / 2; ++m) {
        float2 x = fma2(fk2, y2[m], c2);
        const bool v0 = active && 2 * m < hlen, v1 = active && 2 * m + 1 < hlen;
        st_pred(out + (lbase + (v0 ? 2 * m : 0) * lstep + oc), x.x, v0);
        st_pred(out + (lbase + (v1 ? 2 * m + 1 : 0) * lstep + oc), x.y, v1);
        x.x = v0 ? x.x : 0.f;
        x.y = v1 ? x.y : 0.f;
        if (do_mass) ps.add(x);
    }
    if (do_mass && active) {
        acc.col_begin();
        acc.s = ps.s.x;
        acc.e = ps.e.x;
        acc.add(ps.s.y);
        acc.e = __fadd_rn(acc.e, ps.e.y);
        acc.col_end();
    }
    return top ? 0 : kc;
}

// ------------------------------------------------------------ grid barrier
// Sense-reversing barrier over all CTAs with a time limit.  On timeout the
// CTA records LB_ETIMEOUT in the status word and returns false; so does
// every CTA that sees a recorded failure while waiting.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, long long timeout_ns,
                                             int32_t *status, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile int32_t *vst = status;
        int ok = 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long t0 = globaltimer_ns();
            long long c0 = clock64();
            unsigned it = 0;
            while (*vgen == gen) {
                if ((++it & 31u) == 0u) {
                    if (*vst != 0) { ok = 0; break; }
                    unsigned long long el = globaltimer_ns() - t0;
                    long long ec = clock64() - c0;
                    if ((long long)el > timeout_ns || ec > 4 * timeout_ns) {
                        atomicCAS(status, 0, (int32_t)LB_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *s_flag = ok && (*vst == 0);
    }
    __syncthreads();
    return *s_flag != 0;
}

// ------------------------------------------------------------ global sums
// Processor 0 folds the per-processor partial sums of step s (of this launch)
// into one Neumaier-compensated FP64 sum per grid, in processor order, and
// appends it to the history ring.  Called after the barrier that ends step s.
template <class TC, int THREADS>
__device__ __forceinline__ void reduce_mass(const StepParams<TC> &p, long long t0, int s) {
    const long long tp = t0 + s;
    if (!(p.mass_every > 0 && ((tp + 1) % p.mass_every) == 0)) return;
    const int par = s & 1;
    const unsigned long long seq = *p.mass_seq;
    for (int gi = threadIdx.x; gi < p.ngrids; gi += THREADS) {
        double sum = 0.0, comp = 0.0;
        for (int b = 0; b < p.nbins; ++b) {
            double v = p.bin_mass[((size_t)par * p.nbins + b) * p.ngrids + gi];
            double tt = sum + v;
            comp += fabs(sum) >= fabs(v) ? (sum - tt) + v : (v - tt) + sum;
            sum = tt;
        }
        double *e = p.mass_hist + ((size_t)(seq % kMassHist) * p.ngrids + gi) * 2;
        e[0] = sum;
        e[1] = comp;
        if (!isfinite(sum + comp)) atomicCAS(p.status, 0, (int32_t)LB_ENUMERIC);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.mass_t[seq % kMassHist] = tp;
        __threadfence();
        *p.mass_seq = seq + 1;
    }
}

// ------------------------------------------------------------ work stealing
// Table mode with stealing: a processor's warps take items from its own
// counter; once it runs dry they scan every processor's remaining count
// (a lane reads up to 8 processors' counts at once) and take the next item
// of the processor with the most left (ties: the lowest index).  Each counter hands out every index once,
// so no item runs twice.  Returns the global item index, or -1 when no
// processor has work left.
template <class TC>
__device__ __forceinline__ int pop_with_stealing(const StepParams<TC> &p, int par, int bin,
                                                 int lane) {
    unsigned *ctr = p.bin_ctr + (size_t)par * p.nbins;
    int c = 0;
    if (lane == 0) c = (int)atomicAdd(&ctr[bin], 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c < p.bin_start[bin + 1] - p.bin_start[bin]) return p.bin_start[bin] + c;
    constexpr int kScan = 8;           // processors per lane read before reducing
    for (int attempt = 0; attempt < 4 * p.nbins + 8; ++attempt) {
        int best_rem = 0, best_v = -1;
        for (int base = 0; base < p.nbins; base += kScan * kWarp) {
            // all of this lane's counts first (independent loads, one
            // latency), then the lane's best, then the warp's
            int rem[kScan];
#pragma unroll
            for (int u = 0; u < kScan; ++u) {
                const int v = base + u * kWarp + lane;
                rem[u] = 0;
                if (v < p.nbins)
                    rem[u] = (p.bin_start[v + 1] - p.bin_start[v]) -
                             (int)*(volatile unsigned *)&ctr[v];
            }
            int lr = 0, vv = p.nbins;
#pragma unroll
            for (int u = 0; u < kScan; ++u)
                if (rem[u] > lr) { lr = rem[u]; vv = base + u * kWarp + lane; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int r2 = __shfl_xor_sync(0xffffffffu, lr, o);
                const int v2 = __shfl_xor_sync(0xffffffffu, vv, o);
                if (r2 > lr || (r2 == lr && v2 < vv)) { lr = r2; vv = v2; }
            }
            if (lr > best_rem) { best_rem = lr; best_v = vv; }
        }
        if (best_rem <= 0) return -1;
        int got = 0;
        if (lane == 0) got = (int)atomicAdd(&ctr[best_v], 1u);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got < p.bin_start[best_v + 1] - p.bin_start[best_v]) return p.bin_start[best_v] + got;
    }
    return -1;
}

// Runtime-nz split item in the smallest bucket of HB, HB - 8, ... levels per
// lane that holds the grid's ceil(nz/2) levels (padding levels cost loads,
// selects and predicated stores, so buckets every 8 levels keep the waste
// near 10 % over nz 32..96).
template <class TS, class TC, int HB, bool JAC = false>
__device__ __forceinline__ int split_rt_bucket(const StepParams<TC> &p, const GridDev &g,
                                               const VPDev &vp, int chunk, long long t, int src,
                                               int lane, bool do_mass, LaneSum<TC> &acc) {
    if constexpr (HB > 8) {
        if ((g.nz + 1) / 2 <= HB - 8)
            return split_rt_bucket<TS, TC, HB - 8, JAC>(p, g, vp, chunk, t, src, lane, do_mass,
                                                        acc);
    }
    return process_item_split_rt<TS, TC, HB, JAC>(p, g, vp, chunk, t, src, lane, do_mass, acc);
}

// Head levels (below S0) of the twin solves: packed pairs (c, c) from the
// kernel parameters, or scalar operations on the per-level constants -- the
// latter for the out-of-line Jacobi item code, where the pairs' registers
// would spill.  The operations per value are the same either way.
template <bool PACKED>
__device__ __forceinline__ float2 twin_head_first(const Coef<float> &cf, float2 y) {
    if constexpr (PACKED) return mul2(y, cf.e2[0]);
    else return f2(y.x * cf.e[0], y.y * cf.e[0]);
}
template <bool PACKED>
__device__ __forceinline__ float2 twin_head_fwd(const Coef<float> &cf, int s, float2 pp, float2 y) {
    if constexpr (PACKED) return fma2(pp, cf.rm2[s], mul2(y, cf.e2[s]));
    else return f2(fmaT(pp.x, cf.rm[s], y.x * cf.e[s]), fmaT(pp.y, cf.rm[s], y.y * cf.e[s]));
}
template <bool PACKED>
__device__ __forceinline__ float2 twin_head_back(const Coef<float> &cf, int s, float2 x1, float2 y) {
    if constexpr (PACKED) return fma2(cf.rm2[s], x1, y);
    else return f2(fmaT(cf.rm[s], x1.x, y.x), fmaT(cf.rm[s], x1.y, y.y));
}

// ------------------------------------------------------------ twin halves
// One lane per column with the twisted factorisation of the split kernels
// inside the lane: y2[s] holds (level s, level NZ-1-s), so both halves'
// eliminations, the middle 2x2 system and both back substitutions run as
// one chain of packed FP32x2 operations -- the same operations, in the same
// order, as the split kernels, on half the instructions, without a shuffle.
// A warp's load and store instructions cover 32 columns of one level (runs
// of 32 columns in the VP's row-major order).  The pivots m_s, r m_s of a
// zero-flux end converge, and from level S0 on their FP32 values are one
// constant pair (the host selects this kernel only when that holds): those
// levels use one coefficient pair held in registers, levels below S0 the
// per-level pairs (c, c) of the kernel parameters.
template <class TS, class TC, int NZ, int S0, bool JAC = false>
__device__ __forceinline__ int process_item_twin(const StepParams<TC> &p, const GridDev &g,
                                                 const VPDev &vp, int chunk, long long t, int src,
                                                 int lane, bool do_mass, LaneSum<TC> &acc) {
    static_assert(sizeof(TS) == 4 && sizeof(TC) == 4, "twin kernels are FP32");
    constexpr int H = NZ / 2;
    static_assert(S0 >= 1 && S0 < H && S0 <= kTwinS0, "converged pivots from level S0");
    const ColGeom cg = col_geom(g, vp, chunk, lane);
    const int plane = g.plane;
    const TS *in = static_cast<const TS *>(g.q[src]);
    TS *out = static_cast<TS *>(g.q[src ^ 1]);
    int kc = kc_at(g, cg.i, cg.j, cg.oc, t);
    if (!cg.active || !g.sweeps_on) kc = 0;

    float2 y2[H];                      // (level s, level NZ-1-s)
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, cg.i, cg.j);
#pragma unroll
        for (int s = 0; s < H; ++s)
            y2[s] = f2(jacobi_level<TS, TC>(g, in, s, NZ, jn),
                       jacobi_level<TS, TC>(g, in, NZ - 1 - s, NZ, jn));
    } else if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int lo = s * plane, hi = (NZ - 1 - s) * plane;
            const float2 a = f2(IO<TS, TC>::ld(in + (lo + cg.oi)), IO<TS, TC>::ld(in + (hi + cg.oi)));
            const float2 b = f2(IO<TS, TC>::ld(in + (lo + cg.oj)), IO<TS, TC>::ld(in + (hi + cg.oj)));
            y2[s] = fma2(wy2, b, mul2(wx2, a));
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? NZ - 1 : 0;
        auto level = [&](int k) {
            float v = fmaT(wy, IO<TS, TC>::ld(in + (k * plane + cg.oj)),
                           wx * IO<TS, TC>::ld(in + (k * plane + cg.oi)));
            v = fmaT(k == kdown ? w0 + wz : w0, IO<TS, TC>::ld(in + (k * plane + cg.oc)), v);
            const int ku = k - sz;
            if (ku >= 0 && ku < NZ) v = fmaT(wz, IO<TS, TC>::ld(in + (ku * plane + cg.oc)), v);
            return v;
        };
#pragma unroll
        for (int s = 0; s < H; ++s) y2[s] = f2(level(s), level(NZ - 1 - s));
    }

    // shift by the column's level H-1 value
    const float cref = kc > 0 ? y2[H - 1].x : 0.f;
    if (kc > 0) {
        const float2 nc = f2(-cref, -cref);
#pragma unroll
        for (int s = 0; s < H; ++s) y2[s] = add2(y2[s], nc);
    }
    const Coef<TC> &cf = p.coef;
    const float2 rminf = f2(cf.rm[S0], cf.rm[S0]);
    int rc = cf.resc_every;
    for (int r = 0; r < kc; ++r) {
        // both halves eliminate toward the middle (from level S0 on the
        // forward multiplier e_s is 1: no multiply)
        float2 pp = twin_head_first<!JAC>(cf, y2[0]);
        y2[0] = pp;
#pragma unroll
        for (int s = 1; s < H; ++s) {
            if (s < S0) {
                pp = twin_head_fwd<!JAC>(cf, s, pp, y2[s]);
            } else {
                pp = fma2(pp, rminf, y2[s]);
            }
            y2[s] = pp;
        }
        // middle: x_own = (p + a p_other) / (1 - a^2)
        y2[H - 1] = f2(fmaT(cf.ifa, pp.y, pp.x) * cf.ifc, fmaT(cf.ifa, pp.x, pp.y) * cf.ifc);
        // both back substitutions outward
#pragma unroll
        for (int s = H - 2; s >= 0; --s) {
            if (s < S0)
                y2[s] = twin_head_back<!JAC>(cf, s, y2[s + 1], y2[s]);
            else
                y2[s] = fma2(rminf, y2[s + 1], y2[s]);
        }
        if (--rc == 0) {
            rc = cf.resc_every;
            const float2 rs = f2(cf.resc, cf.resc);
#pragma unroll
            for (int s = 0; s < H; ++s) y2[s] = mul2(y2[s], rs);
        }
    }

    if (cg.active) {
        const float2 c2 = f2(cref, cref), fk2 = f2(cf.f[kc], cf.f[kc]);
        PairSum ps;
        if (do_mass) ps.begin();
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const float2 v = fma2(fk2, y2[s], c2);
            out[s * plane + cg.oc] = v.x;
            out[(NZ - 1 - s) * plane + cg.oc] = v.y;
            if (do_mass) ps.add(v);
        }
        if (do_mass) {
            acc.col_begin();
            acc.s = ps.s.x;
            acc.e = ps.e.x;
            acc.add(ps.s.y);
            acc.e = __fadd_rn(acc.e, ps.e.y);
            acc.col_end();
        }
    }
    return kc;
}

// Twin halves for grids of any nz >= 2 (several grids of different nz in
// one launch): pair s holds (level s, level nz-1-s) for s < HMAX; the lower
// half has hb = ceil(nz/2) levels, the upper ht = floor(nz/2), so each
// component of a pair is masked at its own half length (for odd nz the
// middle level belongs to the lower half only).  Same operations per value,
// in the same order, as the runtime-nz split kernels: clamped loads, selects
// instead of length-dependent branches, predicated stores.
template <class TS, class TC, int HMAX, int S0, bool JAC = false>
__device__ __forceinline__ int process_item_twin_rt(const StepParams<TC> &p, const GridDev &g,
                                                    const VPDev &vp, int chunk, long long t,
                                                    int src, int lane, bool do_mass,
                                                    LaneSum<TC> &acc) {
    static_assert(sizeof(TS) == 4 && sizeof(TC) == 4, "twin kernels are FP32");
    static_assert(HMAX >= 1 && S0 >= 1 && S0 <= kTwinS0, "bucket");
    const ColGeom cg = col_geom(g, vp, chunk, lane);
    const int plane = g.plane, nz = g.nz;
    const int hb = (nz + 1) / 2, ht = nz / 2;
    const TS *in = static_cast<const TS *>(g.q[src]);
    TS *out = static_cast<TS *>(g.q[src ^ 1]);
    int kc = kc_at(g, cg.i, cg.j, cg.oc, t);
    if (!cg.active || !g.sweeps_on) kc = 0;

    float2 y2[HMAX];
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, cg.i, cg.j);
#pragma unroll
        for (int s = 0; s < HMAX; ++s) {
            const float vl = jacobi_level<TS, TC>(g, in, min(s, hb - 1), nz, jn);
            const float vh = jacobi_level<TS, TC>(g, in, nz - 1 - min(s, ht - 1), nz, jn);
            y2[s] = f2(s < hb ? vl : 0.f, s < ht ? vh : 0.f);
        }
    } else if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int s = 0; s < HMAX; ++s) {
            const int lo = min(s, hb - 1) * plane, hi = (nz - 1 - min(s, ht - 1)) * plane;
            const float2 a = f2(IO<TS, TC>::ld(in + (lo + cg.oi)), IO<TS, TC>::ld(in + (hi + cg.oi)));
            const float2 b = f2(IO<TS, TC>::ld(in + (lo + cg.oj)), IO<TS, TC>::ld(in + (hi + cg.oj)));
            const float2 v = fma2(wy2, b, mul2(wx2, a));
            y2[s] = f2(s < hb ? v.x : 0.f, s < ht ? v.y : 0.f);
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? nz - 1 : 0;
        auto level = [&](int k) {
            const float cc = IO<TS, TC>::ld(in + (k * plane + cg.oc));
            const float a = IO<TS, TC>::ld(in + (k * plane + cg.oi));
            const float b = IO<TS, TC>::ld(in + (k * plane + cg.oj));
            float v = fmaT(wy, b, wx * a);
            v = fmaT(k == kdown ? w0 + wz : w0, cc, v);
            const int ku = k - sz;
            const int kuc = ku < 0 ? 0 : (ku >= nz ? nz - 1 : ku);
            const float u = IO<TS, TC>::ld(in + (kuc * plane + cg.oc));
            return (ku >= 0 && ku < nz) ? fmaT(wz, u, v) : v;
        };
#pragma unroll
        for (int s = 0; s < HMAX; ++s) {
            const float vl = level(min(s, hb - 1)), vh = level(nz - 1 - min(s, ht - 1));
            y2[s] = f2(s < hb ? vl : 0.f, s < ht ? vh : 0.f);
        }
    }

    // shift by the column's level hb-1 value (the lower half's last)
    float last = 0.f;
#pragma unroll
    for (int s = 0; s < HMAX; ++s) last = s == hb - 1 ? y2[s].x : last;
    const float cref = kc > 0 ? last : 0.f;
    if (kc > 0) {
        const float2 nc = f2(-cref, -cref);
#pragma unroll
        for (int s = 0; s < HMAX; ++s) y2[s] = add2(y2[s], nc);
    }
    const Coef<TC> &cf = p.coef;
    const float2 rminf = f2(cf.rm[S0], cf.rm[S0]);
    int rc = cf.resc_every;
    for (int r = 0; r < kc; ++r) {
        float2 pp = twin_head_first<!JAC>(cf, y2[0]);
        y2[0] = pp;
#pragma unroll
        for (int s = 1; s < HMAX; ++s) {
            float2 np;
            if (s < S0)
                np = twin_head_fwd<!JAC>(cf, s, pp, y2[s]);
            else
                np = fma2(pp, rminf, y2[s]);
            const bool inl = s < hb, inh = s < ht;
            y2[s] = f2(inl ? np.x : y2[s].x, inh ? np.y : y2[s].y);
            pp = f2(inl ? np.x : pp.x, inh ? np.y : pp.y);
        }
        // middle: pp holds the last eliminated value of each half
        const float xl = fmaT(g.ifa_b_f, pp.y, pp.x) * g.ifc_bt_f;
        const float xh = fmaT(g.ifa_t_f, pp.x, pp.y) * g.ifc_bt_f;
        y2[HMAX - 1] = f2(hb == HMAX ? xl : y2[HMAX - 1].x, ht == HMAX ? xh : y2[HMAX - 1].y);
#pragma unroll
        for (int s = HMAX - 2; s >= 0; --s) {
            float2 bk;
            if (s < S0)
                bk = twin_head_back<!JAC>(cf, s, y2[s + 1], y2[s]);
            else
                bk = fma2(rminf, y2[s + 1], y2[s]);
            y2[s] = f2(s == hb - 1 ? xl : (s < hb - 1 ? bk.x : y2[s].x),
                       s == ht - 1 ? xh : (s < ht - 1 ? bk.y : y2[s].y));
        }
        if (--rc == 0) {
            rc = cf.resc_every;
            const float2 rs = f2(cf.resc, cf.resc);
#pragma unroll
            for (int s = 0; s < HMAX; ++s) y2[s] = mul2(y2[s], rs);
        }
    }

    const float2 c2 = f2(cref, cref), fk2 = f2(cf.f[kc], cf.f[kc]);
    PairSum ps;
    if (do_mass) ps.begin();
#pragma unroll
    for (int s = 0; s < HMAX; ++s) {
        float2 x = fma2(fk2, y2[s], c2);
        const bool vl = cg.active && s < hb, vh = cg.active && s < ht;
        st_pred(out + ((vl ? s : 0) * plane + cg.oc), x.x, vl);
        st_pred(out + ((nz - 1 - (vh ? s : 0)) * plane + cg.oc), x.y, vh);
        x.x = vl ? x.x : 0.f;
        x.y = vh ? x.y : 0.f;
        if (do_mass) ps.add(x);
    }
    if (do_mass && cg.active) {
        acc.col_begin();
        acc.s = ps.s.x;
        acc.e = ps.e.x;
        acc.add(ps.s.y);
        acc.e = __fadd_rn(acc.e, ps.e.y);
        acc.col_end();
    }
    return kc;
}

// Runtime-nz twin item in the smallest bucket of HB, HB - 8, ... pairs that
// holds the grid's ceil(nz/2) levels.
template <class TS, class TC, int HB, bool JAC = false>
__device__ __forceinline__ int twin_rt_bucket(const StepParams<TC> &p, const GridDev &g,
                                              const VPDev &vp, int chunk, long long t, int src,
                                              int lane, bool do_mass, LaneSum<TC> &acc) {
    if constexpr (HB > 8) {
        if ((g.nz + 1) / 2 <= HB - 8)
            return twin_rt_bucket<TS, TC, HB - 8, JAC>(p, g, vp, chunk, t, src, lane, do_mass, acc);
    }
    return process_item_twin_rt<TS, TC, HB, (kTwinS0 < HB ? kTwinS0 : HB), JAC>(
        p, g, vp, chunk, t, src, lane, do_mass, acc);
}

// ------------------------------------------------------------ paired warps
// Split columns on two warps: a work item is a PW x (32 / PW) tile of 32
// columns (PW = 16); lane l of the lower warp holds levels 0..H-1 of
// column l, lane l of the upper warp levels NZ-1..H of the same column (the twisted
// factorisation of the split kernels, with the halves on two warps instead
// of two half-warps).  Every load and store instruction of a warp then
// covers 32 columns of one level where the half-warp split touches two
// levels, 16 columns each; on the 1024 x 1024 x 96 field the memory-only
// rate of the load-compute-store pattern is 5.2 TB/s for 16 x 2 tiles
// against 3.3 TB/s for the half-warp split.  The wider tile idles more
// lanes at the edges of VPs whose widths are not multiples of 16; it runs
// when threads_hint asks for it.  The middle exchange of each solve and the
// column's reference value go through shared memory, with a
// named barrier of the pair's 64 threads.  Both warps hold the same 32
// columns, so they see the same k_c values and the same sweep count and
// reach every barrier together.
struct PairXch {
    float mid[2][2][kWarp];   // [solve parity][half][lane]: last eliminated value
    float ref[kWarp];         // the column's level H-1 value (lower warp)
    int item;                 // work item popped by the lower warp, -1: none
};

__device__ __forceinline__ void pair_sync(int id) {
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Returns the column's k_c on the lower warp, 0 on the upper one.
template <class TS, class TC, int NZ, int PW, bool JAC = false>
__device__ __forceinline__ int process_item_pair(const StepParams<TC> &p, const GridDev &g,
                                                 const VPDev &vp, int chunk, long long t, int src,
                                                 int lane, int top, int bar_id, PairXch &x,
                                                 bool do_mass, LaneSum<TC> &acc) {
    static_assert(sizeof(TS) == 4 && sizeof(TC) == 4, "paired split kernels are FP32");
    constexpr int H = NZ / 2;
    static_assert(H % 2 == 0, "levels are processed in pairs");
    constexpr int PH = kWarp / PW;
    static_assert(PW * PH == kWarp, "a tile is one column per lane");
    const int tiles_x = (vp.w + PW - 1) / PW;
    const int ty = chunk / tiles_x, tx = chunk - ty * tiles_x;
    const int xi = tx * PW + (lane % PW), yi = ty * PH + lane / PW;
    const bool active = xi < vp.w && yi < vp.h;
    const int i = vp.x0 + (xi < vp.w ? xi : vp.w - 1);
    const int j = vp.y0 + (yi < vp.h ? yi : vp.h - 1);
    int im = i - g.sx, jm = j - g.sy;
    im = im < 0 ? im + g.nx : (im >= g.nx ? im - g.nx : im);
    jm = jm < 0 ? jm + g.ny : (jm >= g.ny ? jm - g.ny : jm);
    const int plane = g.plane;
    const int oc = j * g.pitch + i, oi = j * g.pitch + im, oj = jm * g.pitch + i;
    const int lbase = top ? (NZ - 1) * plane : 0;
    const int lstep = top ? -plane : plane;
    const TS *in = static_cast<const TS *>(g.q[src]);
    TS *out = static_cast<TS *>(g.q[src ^ 1]);
    int kc = kc_at(g, i, j, oc, t);
    if (!active || !g.sweeps_on) kc = 0;

    float2 y2[H / 2];
    float *y = reinterpret_cast<float *>(y2);
    const float wx = wgt<float>(g, 1), wy = wgt<float>(g, 2);
    if constexpr (JAC) {
        const JacNbr jn = jac_nbr(g, i, j);
#pragma unroll
        for (int s = 0; s < H; ++s) y[s] = jacobi_level<TS, TC>(g, in, top ? NZ - 1 - s : s, NZ, jn);
    } else if (g.xy_only) {
        const float2 wx2 = f2(wx, wx), wy2 = f2(wy, wy);
#pragma unroll
        for (int m = 0; m < H / 2; ++m) {
            const int off0 = lbase + (2 * m) * lstep, off1 = off0 + lstep;
            const float2 a = f2(IO<TS, TC>::ld(in + (off0 + oi)), IO<TS, TC>::ld(in + (off1 + oi)));
            const float2 b = f2(IO<TS, TC>::ld(in + (off0 + oj)), IO<TS, TC>::ld(in + (off1 + oj)));
            y2[m] = fma2(wy2, b, mul2(wx2, a));
        }
    } else {
        const float w0 = wgt<float>(g, 0), wz = wgt<float>(g, 3);
        const int sz = g.sz;
        const int kdown = sz >= 0 ? NZ - 1 : 0;
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int k = top ? NZ - 1 - s : s;
            const int off = lbase + s * lstep;
            float c = IO<TS, TC>::ld(in + (off + oc));
            float a = IO<TS, TC>::ld(in + (off + oi));
            float b = IO<TS, TC>::ld(in + (off + oj));
            float v = fmaT(wy, b, wx * a);
            v = fmaT(k == kdown ? w0 + wz : w0, c, v);
            const int ku = k - sz;
            if (ku >= 0 && ku < NZ) v = fmaT(wz, IO<TS, TC>::ld(in + (ku * plane + oc)), v);
            y[s] = v;
        }
    }

    // shift by the column's level H-1 value (held by the lower warp)
    if (!top) x.ref[lane] = y[H - 1];
    pair_sync(bar_id);
    const float cref = kc > 0 ? x.ref[lane] : 0.f;
    if (kc > 0) {
        const float2 nc = f2(-cref, -cref);
#pragma unroll
        for (int m = 0; m < H / 2; ++m) y2[m] = add2(y2[m], nc);
    }
    const Coef<TC> &cf = p.coef;
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)kc);
    int rc = cf.resc_every;
    for (int r = 0; r < kmax; ++r) {
        const bool act = r < kc;
        if (act) {
            float pp = y[0] * cf.e[0];
            y[0] = pp;
#pragma unroll
            for (int s = 1; s < H; ++s) {
                pp = fmaT(pp, cf.rm[s], y[s] * cf.e[s]);
                y[s] = pp;
            }
        }
        x.mid[r & 1][top][lane] = y[H - 1];
        pair_sync(bar_id);
        const float other = x.mid[r & 1][top ^ 1][lane];
        if (act) {
            y[H - 1] = fmaT(cf.ifa, other, y[H - 1]) * cf.ifc;
#pragma unroll
            for (int s = H - 2; s >= 0; --s) y[s] = fmaT(cf.rm[s], y[s + 1], y[s]);
            if (--rc == 0) {
                rc = cf.resc_every;
                const float2 rs = f2(cf.resc, cf.resc);
#pragma unroll
                for (int m = 0; m < H / 2; ++m) y2[m] = mul2(y2[m], rs);
            }
        }
    }

    if (active) {
        const float2 c2 = f2(cref, cref), fk2 = f2(cf.f[kc], cf.f[kc]);
        PairSum ps;
        if (do_mass) ps.begin();
#pragma unroll
        for (int m = 0; m < H / 2; ++m) {
            const float2 v = fma2(fk2, y2[m], c2);
            out[lbase + (2 * m) * lstep + oc] = v.x;
            out[lbase + (2 * m + 1) * lstep + oc] = v.y;
            if (do_mass) ps.add(v);
        }
        if (do_mass) {
            acc.col_begin();
            acc.s = ps.s.x;
            acc.e = ps.e.x;
            acc.add(ps.s.y);
            acc.e = __fadd_rn(acc.e, ps.e.y);
            acc.col_end();
        }
    }
    return top ? 0 : kc;
}

// Next work item of a warp (processor tables, stealing or atomic queue),
// -1 when none is left this step.
template <class TC>
__device__ __forceinline__ int pop_item(const StepParams<TC> &p, int s, int bin, int lane, int *s_ctr,
                                        int ibeg, int iend) {
    if (p.steal && !p.queue_mode) return pop_with_stealing(p, s & 1, bin, lane);
    int c = 0;
    if (lane == 0) c = p.queue_mode ? (int)atomicAdd(&p.qhead[s & 1], 1u) : atomicAdd(s_ctr, 1);
    c = __shfl_sync(0xffffffffu, c, 0) + ibeg;
    return c < iend ? c : -1;
}

// ------------------------------------------------------------ item dispatch
template <class TC>
struct ItemResult {
    int kc;
    LaneSum<TC> acc;
};

// One work item of the kernel variant, with the advection (JAC false) or the
// Jacobi form of the dynamics phase.
template <class TS, class TC, int NZ, bool EXACT, int NZLO, bool SPLIT, bool TWIN, bool JAC>
__device__ __forceinline__ int run_item(const StepParams<TC> &p, const GridDev &g, const VPDev &vp,
                                        int chunk, long long t, int src, int lane, bool do_mass,
                                        LaneSum<TC> &acc) {
    if constexpr (TWIN && EXACT)
        return process_item_twin<TS, TC, NZ, kTwinS0, JAC>(p, g, vp, chunk, t, src, lane, do_mass,
                                                           acc);
    else if constexpr (TWIN)
        return twin_rt_bucket<TS, TC, NZ / 2, JAC>(p, g, vp, chunk, t, src, lane, do_mass, acc);
    else if constexpr (SPLIT && EXACT)
        return process_item_split<TS, TC, NZ, JAC>(p, g, vp, chunk, t, src, lane, do_mass, acc);
    else if constexpr (SPLIT)
        // per item (one grid, warp-uniform): the smallest half-length bucket
        // (multiples of 8 levels) that holds the grid's ceil(nz/2) levels
        return split_rt_bucket<TS, TC, NZ / 2, JAC>(p, g, vp, chunk, t, src, lane, do_mass, acc);
    else
        return process_item<TS, TC, NZ, EXACT, NZLO, JAC>(p, g, vp, chunk, t, src, lane, do_mass,
                                                         acc);
}

// Items of grids with the Jacobi dynamics run through out-of-line copies of
// the item code, so that the advection path keeps its own register
// allocation (arguments and the lane sums by value: no address of the
// caller's registers is taken).
template <class TS, class TC, int NZ, bool EXACT, int NZLO, bool SPLIT, bool TWIN>
__device__ __noinline__ ItemResult<TC> run_item_jacobi(const StepParams<TC> &p, const GridDev *g,
                                                       VPDev vp, int chunk, long long t, int src,
                                                       int lane, bool do_mass, LaneSum<TC> acc) {
    ItemResult<TC> r;
    r.kc = run_item<TS, TC, NZ, EXACT, NZLO, SPLIT, TWIN, true>(p, *g, vp, chunk, t, src, lane,
                                                               do_mass, acc);
    r.acc = acc;
    return r;
}

template <class TS, class TC, int NZ, int PW>
__device__ __noinline__ ItemResult<TC> run_pair_jacobi(const StepParams<TC> &p, const GridDev *g,
                                                       VPDev vp, int chunk, long long t, int src,
                                                       int lane, int top, int bar_id, PairXch *x,
                                                       bool do_mass, LaneSum<TC> acc) {
    ItemResult<TC> r;
    r.kc = process_item_pair<TS, TC, NZ, PW, true>(p, *g, vp, chunk, t, src, lane, top, bar_id, *x,
                                                  do_mass, acc);
    r.acc = acc;
    return r;
}

// ------------------------------------------------------------ the kernel
// MINB: CTAs that must fit on one SM (processors sharing an SM), which caps
// the registers per thread at 65536 / (THREADS * MINB).
template <class TS, class TC, int NZ, bool EXACT, int NZLO, int THREADS, bool SPLIT, int PAIRW,
          bool TWIN, int MINB = 1>
__global__ void __launch_bounds__(THREADS, MINB)
lb_step_kernel(const __grid_constant__ StepParams<TC> p) {
    constexpr bool PAIR = PAIRW > 0;
    static_assert(!TWIN || (!SPLIT && !PAIR), "twin kernels: one lane per column");
    static_assert(!PAIR || (SPLIT && EXACT && THREADS % 64 == 0 && THREADS / 64 <= 15),
                  "paired warps: exact split columns, at most 15 pairs (named barriers 1..15)");
    extern __shared__ double s_mass[];          // [warps][ngrids]
    __shared__ PairXch s_pair[PAIR ? THREADS / 64 : 1];
    __shared__ int s_ctr;
    __shared__ int s_flag;
    __shared__ unsigned long long s_t0, s_tend;
    constexpr int kWarps = THREADS / kWarp;
    const int bin = blockIdx.x;
    const int warp = threadIdx.x / kWarp;
    const int lane = threadIdx.x % kWarp;

    if (threadIdx.x == 0) {
        p.bin_smid[bin] = smid();
        p.bin_cal[4 * bin + 0] = (long long)globaltimer_ns();
        p.bin_cal[4 * bin + 1] = clock64();
    }
    const int ibeg = p.queue_mode ? 0 : p.bin_start[bin];
    const int iend = p.queue_mode ? p.nitems : p.bin_start[bin + 1];
    // step index and buffer parity: kernel parameters, or the device clock
    // (graph replays: parameters are frozen at capture, the clock is not)
    const long long t0 = p.dclock ? p.dclock[0] : p.t0;
    const int parity0 = p.dclock ? (int)p.dclock[1] : p.parity0;

    for (int s = 0; s < p.nsteps; ++s) {
        const long long t = t0 + s;
        const int src = (parity0 + s) & 1;
        const bool do_mass = p.mass_every > 0 && ((t + 1) % p.mass_every) == 0;

        // reduce the previous step's per-processor sums (processor 0 only)
        if (bin == 0 && s > 0) reduce_mass<TC, THREADS>(p, t0, s - 1);

        if (threadIdx.x == 0) {
            s_ctr = 0;
            s_tend = 0ull;
            s_t0 = (unsigned long long)clock64();
            if (bin == 0) p.qhead[(s + 1) & 1] = 0u;
            // next step's counter: nobody touches it before this step's barrier
            if (p.steal) p.bin_ctr[(size_t)((s + 1) & 1) * p.nbins + bin] = 0u;
        }
        if (do_mass)
            for (int n = threadIdx.x; n < kWarps * p.ngrids; n += THREADS) s_mass[n] = 0.0;
        __syncthreads();

        LaneSum<TC> acc;
        int cur_grid = -1;
        if constexpr (PAIR) {
            // the lower warp of each pair pops; both process the item
            const int top = warp & 1, bar_id = 1 + (warp >> 1);
            PairXch &x = s_pair[warp >> 1];
            for (;;) {
                if (!top) {
                    const int c = pop_item(p, s, bin, lane, &s_ctr, ibeg, iend);
                    if (lane == 0) x.item = c;
                }
                pair_sync(bar_id);
                const int c = x.item;
                if (c < 0) break;
                const int2 it = p.items[c];
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
                const long long c0 = clock64();
                constexpr int PW = PAIR ? PAIRW : 16;
                int kc;
                if (g.jacobi) {
                    const ItemResult<TC> r = run_pair_jacobi<TS, TC, NZ, PW>(
                        p, &g, vp, it.y, t, src, lane, top, bar_id, &x, do_mass, acc);
                    kc = r.kc;
                    acc = r.acc;
                } else {
                    kc = process_item_pair<TS, TC, NZ, PW>(p, g, vp, it.y, t, src, lane, top, bar_id,
                                                            x, do_mass, acc);
                }
                __syncwarp();
                const long long c1 = clock64();
                const unsigned ksum = __reduce_add_sync(0xffffffffu, (unsigned)kc);
                if (lane == 0 && !top) {
                    atomicAdd(&p.vp_cycles[it.x], (unsigned long long)(c1 - c0));
                    if (p.sweeps) atomicAdd(p.sweeps, (unsigned long long)ksum * (unsigned)g.nz);
                }
            }
        } else for (;;) {
            // serial measurement steps: only the first serial_warps warps work
            if (p.serial_warps > 0 && warp >= p.serial_warps) break;
            int c = 0;
            if (p.steal && !p.queue_mode) {
                c = pop_with_stealing(p, s & 1, bin, lane);
                if (c < 0) break;
            } else {
                if (lane == 0)
                    c = p.queue_mode ? (int)atomicAdd(&p.qhead[s & 1], 1u) : atomicAdd(&s_ctr, 1);
                c = __shfl_sync(0xffffffffu, c, 0) + ibeg;
                if (c >= iend) break;
            }
            const int2 it = p.items[c];
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
            long long c0 = clock64();
            int kc;
            if (g.jacobi) {
                const ItemResult<TC> r = run_item_jacobi<TS, TC, NZ, EXACT, NZLO, SPLIT, TWIN>(
                    p, &g, vp, it.y, t, src, lane, do_mass, acc);
                kc = r.kc;
                acc = r.acc;
            } else {
                kc = run_item<TS, TC, NZ, EXACT, NZLO, SPLIT, TWIN, false>(p, g, vp, it.y, t, src,
                                                                            lane, do_mass, acc);
            }
            __syncwarp();
            long long c1 = clock64();
            // cell-sweep updates actually performed: sum of k_c * nz over the item
            const unsigned ksum = __reduce_add_sync(0xffffffffu, (unsigned)kc);
            if (lane == 0) {
                atomicAdd(&p.vp_cycles[it.x], (unsigned long long)(c1 - c0));
                if (p.sweeps) atomicAdd(p.sweeps, (unsigned long long)ksum * (unsigned)g.nz);
            }
        }
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
        if (!grid_barrier(p.bar, gridDim.x, p.timeout_ns, p.status, &s_flag)) return;
    }

    // the last step's sums; advance the device clock (every CTA read it
    // before the first barrier, so processor 0 may now overwrite it)
    if (bin == 0 && p.nsteps > 0) {
        reduce_mass<TC, THREADS>(p, t0, p.nsteps - 1);
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

template <class TS, class TC, int NZ, bool EXACT, int NZLO, int THREADS, bool SPLIT = false,
          int PAIRW = 0, bool TWIN = false, int MINB = 1>
inline KernelInfo kernel_entry() {
    static_assert(!SPLIT || NZ % 4 == 0, "split kernels hold nz/2 levels in register pairs");
    constexpr bool PAIR = PAIRW > 0;
    KernelInfo k;
    k.fn = (const void *)&lb_step_kernel<TS, TC, NZ, EXACT, NZLO, THREADS, SPLIT, PAIRW, TWIN, MINB>;
    k.df_fn = nullptr;
    k.threads = THREADS;
    k.nz_variant = NZ;
    k.exact = EXACT ? 1 : 0;
    // twin kernels use the split kernels' coefficient tables
    k.split = (SPLIT || TWIN) ? 1 : 0;
    k.twin_s0 = TWIN ? kTwinS0 : 0;
    k.cols_per_item = (SPLIT && !PAIR) ? kWarp / 2 : kWarp;
    k.tile_w = PAIR ? PAIRW : (SPLIT ? kTileW : 0);
    k.tile_h = PAIR ? kWarp / PAIRW : (SPLIT ? kTileH : 0);
    k.tma_slots = 0;
    k.tma_slot_bytes = 0;
    return k;
}

}  // namespace lbk

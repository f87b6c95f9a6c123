// batch.cu - many independent 2D MLS pressure-Poisson systems (Sec. 3.3,
// Eq. (21)) built and solved together.
//
// The systems are stored back to back: system i owns DPs [off_i, off_i + N_i)
// of every per-DP array, its rows are the [slot][N_i] block at 9 off_i, and
// its positions the [2][N_i] block at 2 off_i.
//
// Solve: one cooperative persistent launch runs Bi-CGSTAB (van der Vorst) on
// every system in lockstep "sweeps".  A sweep has three slots separated by
// grid barriers; in each slot the tiles of all systems still running are
// split evenly over the CTAs (a CTA takes a contiguous range of the
// (system, tile) work list, which is rebuilt over the systems still running
// at the end of every sweep, so converged systems free their CTAs at once).
// Each system is in one of two modes for a whole sweep:
//   ITER    slot A  p = r + beta (p - omega v), v = A p      -> alpha
//           slot B  s = r - alpha v, t = A s                  -> omega
//           slot C  x += alpha p + omega s, r = s - omega t   -> beta, tests
//   UPDATE  slot A  (MIXED) x64 += x32, x32 = 0
//           slot B  r = b - A64 x64 (FP64 residual)           -> converged?
//                   else restart the recursion from it
// so the true-residual (reliable) updates of the mixed solve cost no extra
// barriers.  Dot products of a system are block-reduced per CTA (FP64, or
// double-float for the FP32 recursion) and added into per-system FP64
// accumulators with atomics; at the barrier, thread j of block 0 finishes
// the reductions of system j, updates its scalars and (end of a sweep)
// rebuilds the work list with a block scan.  Every wait is bounded: a
// barrier that gives up sets phase_err and the launch ends.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "krylov_common.cuh"

namespace mcd {
namespace batch {

// Geometry of one system for the solver (tile counts depend on the tiling).
struct BGeo {
    int n0, n1, per0, per1;
    int64_t N, off;
    int tiles_x, ntiles;
};

enum { MODE_SKIP = 0, MODE_ITER = 1, MODE_UPDATE = 2 };

// Krylov scalars of one system (owned by thread (system index) of block 0
// at the barriers).
struct BScal {
    double rho, alpha, omega, beta, rhat2, tol2, rr, rr64, bb64, rr_last;
    float alpha_f, omega_f, beta_f, pad_f;
    int iter, max_iter;
    int done;      // 0 running, 1 converged, 2 max_iter, 3 breakdown, 4 nonfinite
    int restart, restarts, s_conv, pending, max_hit, parity, mode;
    int updates;   // true-residual updates after the first
    int it_last;   // iteration of the last true residual
    int discard;   // MIXED: the cycle diverged: drop its correction (UPDATE slot A)
    int no_replace;   // a replaced recursion diverged: restart at every later update
    int discarded;    // cycles dropped
};

struct BState {
    int n_active;      // systems still running
    int phase_err;     // a barrier gave up
    int list;          // which of the two work lists is current
    int pad;
    int64_t M;         // tiles of the systems still running
    int64_t sweeps;    // sweeps run (all launches)
};

struct BArgs {
    int nsys;
    const BGeo *geo;
    const int8_t *kind;
    const void *row;          // recursion rows (FP32 difference form or FP64)
    const double *row64;      // FP64 rows (true residual)
    const double *b;
    double *x64;
    void *x, *r, *rh, *p0, *p1, *v0, *v1, *s, *t;
    float *xlo;               // MIXED: low word of the double-float correction (x, xlo)
    BScal *sc;
    double *acc;              // [3 slots][nsys][4] FP64 accumulators
    int *active;              // [2][nsys] work lists (system ids)
    int64_t *prefix;          // [2][nsys + 1] tile prefix sums of the lists
    BState *state;
    GridBarrier *bar;
    int mixed;
    double tol2_factor;       // tol^2
    double update2;           // MIXED: update once rr <= update2 rr_last
    int replace;              // MIXED: residual replacement until a cycle diverges (adaptive)
    int stall;                // MIXED: update after this many iterations without one
    double eps_breakdown;
    int budget;               // sweeps this launch may run
    long long spin_limit;
};

template <int R> struct BT {
    static constexpr int X = 32, TY = 8, Y = 8 * R, HX = X + 2, HY = Y + 2, H = HX * HY;
    static constexpr int HN = (H + 255) / 256;
};

__device__ __forceinline__ int64_t bt_halo(const BGeo &g, int h, int x0, int y0, int hx_n) {
    const int hx = h % hx_n, hy = h / hx_n;
    const int gx = wrap_clamp(x0 + hx - 1, g.n0, g.per0);
    const int gy = wrap_clamp(y0 + hy - 1, g.n1, g.per1);
    return (int64_t)gx + (int64_t)g.n0 * gy;
}

template <int R>
__device__ __forceinline__ int64_t bt_dp(const BGeo &g, int tid, int q, int x0, int y0, int &lx, int &ly) {
    lx = tid % BT<R>::X;
    ly = tid / BT<R>::X + q * BT<R>::TY;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= g.n0 || gy >= g.n1) return -1;
    return (int64_t)gx + (int64_t)g.n0 * gy;
}

template <int R>
__device__ __forceinline__ void bt_origin(const BGeo &g, int64_t t, int &x0, int &y0) {
    const int tx = (int)(t % g.tiles_x), ty = (int)(t / g.tiles_x);
    x0 = tx * BT<R>::X;
    y0 = ty * BT<R>::Y;
}

// ---- per-tile work ---------------------------------------------------------
// Pointers are the system's own (already offset); rows are [9][N].

template <typename T, int R>
__device__ void tile_a(const BGeo &g, int64_t t, T *tile, const T *row, const T *r, T *rhat, const T *p_old,
                       const T *v_old, T *p_new, T *v_new, T beta, T omega, int restart, DotAcc<T> (&dot)[3]) {
    using B = BT<R>;
    const int tid = threadIdx.x;
    int x0, y0;
    bt_origin<R>(g, t, x0, y0);
    int64_t k[R];
    int lx[R], ly[R];
    T w[R][9];
    T rh[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        k[q] = bt_dp<R>(g, tid, q, x0, y0, lx[q], ly[q]);
        load_row<9, T>(row, g.N, k[q], w[q]);
        rh[q] = (!restart && k[q] >= 0) ? __ldcg(rhat + k[q]) : (T)0;
    }
    T hr[B::HN], hp[B::HN], hv[B::HN];
#pragma unroll
    for (int u = 0; u < B::HN; ++u) {
        const int h = tid + u * 256;
        hr[u] = hp[u] = hv[u] = (T)0;
        if (h < B::H) {
            const int64_t j = bt_halo(g, h, x0, y0, B::HX);
            hr[u] = __ldcg(r + j);
            if (!restart) {
                hp[u] = __ldcg(p_old + j);
                hv[u] = __ldcg(v_old + j);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < B::HN; ++u) {
        const int h = tid + u * 256;
        if (h < B::H) tile[h] = restart ? hr[u] : hr[u] + beta * (hp[u] - omega * hv[u]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (k[q] < 0) continue;
        const T pk = tile[(lx[q] + 1) + B::HX * (ly[q] + 1)];
        p_new[k[q]] = pk;
        T rq = rh[q];
        if (restart) {
            rq = pk;
            rhat[k[q]] = rq;
            dot[1].add(rq, pk);
            dot[2].add(rq, rq);
        }
        const T vk = stencil_apply<2, T>(w[q], tile, lx[q], ly[q], 0);
        v_new[k[q]] = vk;
        dot[0].add(rq, vk);
    }
    __syncthreads();
}

template <typename T, int R>
__device__ void tile_b(const BGeo &g, int64_t t, T *tile, const T *row, const T *r, const T *v, T *s_out,
                       T *t_out, T alpha, DotAcc<T> (&dot)[3]) {
    using B = BT<R>;
    const int tid = threadIdx.x;
    int x0, y0;
    bt_origin<R>(g, t, x0, y0);
    int64_t k[R];
    int lx[R], ly[R];
    T w[R][9];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        k[q] = bt_dp<R>(g, tid, q, x0, y0, lx[q], ly[q]);
        load_row<9, T>(row, g.N, k[q], w[q]);
    }
    T hr[B::HN], hv[B::HN];
#pragma unroll
    for (int u = 0; u < B::HN; ++u) {
        const int h = tid + u * 256;
        hr[u] = hv[u] = (T)0;
        if (h < B::H) {
            const int64_t j = bt_halo(g, h, x0, y0, B::HX);
            hr[u] = __ldcg(r + j);
            hv[u] = __ldcg(v + j);
        }
    }
#pragma unroll
    for (int u = 0; u < B::HN; ++u) {
        const int h = tid + u * 256;
        if (h < B::H) tile[h] = hr[u] - alpha * hv[u];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (k[q] < 0) continue;
        const T sk = tile[(lx[q] + 1) + B::HX * (ly[q] + 1)];
        s_out[k[q]] = sk;
        const T tk = stencil_apply<2, T>(w[q], tile, lx[q], ly[q], 0);
        t_out[k[q]] = tk;
        dot[0].add(tk, sk);
        dot[1].add(tk, tk);
        dot[2].add(sk, sk);
    }
    __syncthreads();
}

template <typename T, int R>
__device__ void tile_c(const BGeo &g, int64_t t, T *x, float *xlo, T *r, const T *rhat, const T *p, const T *s,
                       const T *tv, T alpha, T omega, int sconv, DotAcc<T> (&dot)[2]) {
    const int tid = threadIdx.x;
    int x0, y0;
    bt_origin<R>(g, t, x0, y0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        int lx, ly;
        const int64_t k = bt_dp<R>(g, tid, q, x0, y0, lx, ly);
        if (k < 0) continue;
        const T xv = __ldcg(x + k), pv = __ldcg(p + k), sv = __ldcg(s + k), tt = __ldcg(tv + k);
        const T hv = __ldcg(rhat + k);
        T rk;
        if constexpr (sizeof(T) == 4) {
            if (xlo) {
                // the correction as a double-float pair: the increments are
                // split exactly and added by TwoSum, so the fold adds an
                // error of order eps^2 |x| rather than eps |x|
                DF acc{xv, __ldcg(xlo + k)};
                df_add_prod(acc, alpha, pv);
                if (!sconv) df_add_prod(acc, omega, sv);
                float hi, lo;
                two_sum_f(acc.hi, acc.lo, hi, lo);
                x[k] = hi;
                xlo[k] = lo;
                rk = sconv ? sv : sv - omega * tt;
                r[k] = rk;
                dot[0].add(hv, rk);
                dot[1].add(rk, rk);
                continue;
            }
        }
        if (sconv) {
            x[k] = xv + alpha * pv;
            rk = sv;
        } else {
            x[k] = xv + alpha * pv + omega * sv;
            rk = sv - omega * tt;
        }
        r[k] = rk;
        dot[0].add(hv, rk);
        dot[1].add(rk, rk);
    }
}

template <typename T, int R>
__device__ void tile_fold(const BGeo &g, int64_t t, double *x64, T *x, float *xlo, bool discard) {
    const int tid = threadIdx.x;
    int x0, y0;
    bt_origin<R>(g, t, x0, y0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        int lx, ly;
        const int64_t k = bt_dp<R>(g, tid, q, x0, y0, lx, ly);
        if (k < 0) continue;
        double add = (double)__ldcg(x + k);
        if (xlo) {
            add += (double)__ldcg(xlo + k);
            xlo[k] = 0.0f;
        }
        if (!discard) x64[k] += add;
        x[k] = (T)0;
    }
}

// r = b - A64 x64 stored in the recursion's precision; dots ||r64||^2 and
// ||b||^2 (FP64), r.r and r^.r of the stored residual.
template <typename T, int R>
__device__ void tile_true_residual(const BGeo &g, int64_t t, const double *row64, const double *b,
                                   const double *x64, T *r, const T *rhat, DotAcc<T> (&rr)[2], double (&d64)[2]) {
    const int tid = threadIdx.x;
    int x0, y0;
    bt_origin<R>(g, t, x0, y0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        int lx, ly;
        const int64_t k = bt_dp<R>(g, tid, q, x0, y0, lx, ly);
        if (k < 0) continue;
        const int gx = x0 + lx, gy = y0 + ly;
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            const int jx = wrap_clamp(gx + s % 3 - 1, g.n0, g.per0);
            const int jy = wrap_clamp(gy + s / 3 - 1, g.n1, g.per1);
            acc += __ldg(row64 + (int64_t)s * g.N + k) * __ldcg(x64 + (int64_t)jx + (int64_t)g.n0 * jy);
        }
        const double bk = b[k];
        const double rk = bk - acc;
        const T rt = (T)rk;
        r[k] = rt;
        d64[0] += rk * rk;
        d64[1] += bk * bk;
        rr[0].add(rt, rt);
        rr[1].add(__ldcg(rhat + k), rt);
    }
}

// ---- reductions, barrier, work list ---------------------------------------

// Block-reduce NV accumulators and add the totals into acc[0..NV-1].
template <typename T, int NV>
__device__ void flush(DotAcc<T> (&d)[NV], double *acc) {
    __shared__ double s_tot[4];
    dot_partials<NV>(d, s_tot, 1, 0);
    if (threadIdx.x == 0)
        for (int q = 0; q < NV; ++q)
            if (s_tot[q] != 0.0) atomicAdd(acc + q, s_tot[q]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) d[q] = DotAcc<T>();
}

__device__ void flush64(double (&v)[2], double *acc) {
    __shared__ double s_tot[2];
    block_partials<2, double>(v, s_tot, 1, 0);
    if (threadIdx.x == 0)
        for (int q = 0; q < 2; ++q)
            if (s_tot[q] != 0.0) atomicAdd(acc + q, s_tot[q]);
    __syncthreads();
    v[0] = v[1] = 0.0;
}

// Grid barrier whose release is preceded by reduce(tid) on all 256 threads
// of block 0.  Returns false if a wait gave up.
template <typename F>
__device__ bool barrier(const BArgs &a, unsigned &epoch, F reduce) {
    __shared__ int s_err;
    const int tid = threadIdx.x;
    ++epoch;
    if (tid == 0) s_err = 0;
    __syncthreads();
    if (tid == 0) st_release(&a.bar->flag[blockIdx.x], epoch);
    if (blockIdx.x == 0) {
        for (int b = tid; b < (int)gridDim.x; b += 256)
            if (!wait_eq(&a.bar->flag[b], epoch, a.spin_limit)) {
                s_err = 1;
                break;
            }
        __syncthreads();
        if (s_err) {
            if (tid == 0) a.state->phase_err = 1;
            return false;
        }
        reduce(tid);
        __syncthreads();
        for (int b = 1 + tid; b < (int)gridDim.x; b += 256)
            st_release(release_word(a.bar, gridDim.x, b), epoch);
    } else if (tid == 0) {
        if (!wait_eq(release_word(a.bar, gridDim.x, blockIdx.x), epoch, a.spin_limit)) {
            s_err = 1;
            a.state->phase_err = 1;
        }
    }
    __syncthreads();
    return !s_err;
}

__device__ __forceinline__ void publish(BScal *c) {
    c->alpha_f = (float)c->alpha;
    c->omega_f = (float)c->omega;
    c->beta_f = (float)c->beta;
}

// Exclusive block scan (256 threads) of (count, tiles); totals returned.
__device__ void scan2(int c, int64_t w, int &cpos, int64_t &wpos, int &ctot, int64_t &wtot) {
    __shared__ int sc_[8];
    __shared__ int64_t sw_[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ci = c;
    int64_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
        const int cu = __shfl_up_sync(0xffffffffu, ci, o);
        const int64_t wu = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) { ci += cu; wi += wu; }
    }
    if (lane == 31) { sc_[warp] = ci; sw_[warp] = wi; }
    __syncthreads();
    int cb = 0;
    int64_t wb = 0;
    ctot = 0;
    wtot = 0;
    for (int q = 0; q < 8; ++q) {
        if (q < warp) { cb += sc_[q]; wb += sw_[q]; }
        ctot += sc_[q];
        wtot += sw_[q];
    }
    cpos = cb + ci - c;
    wpos = wb + wi - w;
    __syncthreads();
}

// Rebuild the work list from the current one (systems not done), on block 0.
__device__ void rebuild_list(const BArgs &a, int na, int cur) {
    const int nxt = cur ^ 1;
    const int *src = a.active + (size_t)cur * a.nsys;
    int *dst = a.active + (size_t)nxt * a.nsys;
    int64_t *pre = a.prefix + (size_t)nxt * (a.nsys + 1);
    int base = 0;
    int64_t wbase = 0;
    for (int c0 = 0; c0 < na; c0 += 256) {
        const int j = c0 + threadIdx.x;
        int keep = 0;
        int64_t tiles = 0;
        int sys = -1;
        if (j < na) {
            sys = src[j];
            if (!a.sc[sys].done) {
                keep = 1;
                tiles = a.geo[sys].ntiles;
            }
        }
        int cpos, ctot;
        int64_t wpos, wtot;
        scan2(keep, tiles, cpos, wpos, ctot, wtot);
        if (keep) {
            dst[base + cpos] = sys;
            pre[base + cpos] = wbase + wpos;
        }
        base += ctot;
        wbase += wtot;
    }
    if (threadIdx.x == 0) {
        pre[base] = wbase;
        a.state->n_active = base;
        a.state->M = wbase;
        a.state->list = nxt;
        a.state->sweeps += 1;
    }
}

// Walk the CTA's share [lo, hi) of the work list; fn(system, first tile,
// end tile) per system segment, in list order.
template <typename F>
__device__ void for_segments(const BArgs &a, int na, int list, int64_t M, F fn) {
    const int *act = a.active + (size_t)list * a.nsys;
    const int64_t *pre = a.prefix + (size_t)list * (a.nsys + 1);
    const int64_t lo = M * (int64_t)blockIdx.x / gridDim.x;
    const int64_t hi = M * (int64_t)(blockIdx.x + 1) / gridDim.x;
    if (lo >= hi) return;
    int l = 0, h = na - 1;   // last j with pre[j] <= lo
    while (l < h) {
        const int m = (l + h + 1) >> 1;
        if (__ldcg(pre + m) <= lo) l = m; else h = m - 1;
    }
    int64_t i = lo;
    for (int j = l; i < hi && j < na; ++j) {
        const int64_t p0 = __ldcg(pre + j), p1 = __ldcg(pre + j + 1);
        const int64_t e = p1 < hi ? p1 : hi;
        if (e > i) fn(__ldcg(act + j), i - p0, e - p0);
        i = e;
    }
}

// Occupancy: the block's tile loop waits on its loads once per tile, so more
// resident blocks hide more of that latency.  The tilings whose registers fit
// 64 per thread without spilling (FP32 with 1 or 2 rows, FP64 with 1) ask for
// four blocks per SM; the others leave the count to the compiler.
template <typename T, int R> struct BatchOcc {
    static constexpr int min_blocks = (R == 1 || (R == 2 && sizeof(T) == 4)) ? 4 : 0;
};

template <typename T, int R>
__global__ void __launch_bounds__(256, BatchOcc<T, R>::min_blocks) bicg_batch(const __grid_constant__ BArgs a) {
    __shared__ T tile[BT<R>::H];
    __shared__ int s_na, s_list, s_err;
    __shared__ long long s_M;
    unsigned epoch = 0;
    const int tid = threadIdx.x;
    const T *row = (const T *)a.row;
    for (int sweep = 0;; ++sweep) {
        if (tid == 0) {
            s_na = vload(&a.state->n_active);
            s_list = vload(&a.state->list);
            s_err = vload(&a.state->phase_err);
            s_M = (long long)vload(&a.state->M);
        }
        __syncthreads();
        const int na = s_na, list = s_list;
        const int64_t M = s_M;
        if (na == 0 || s_err || sweep >= a.budget) return;
        double *accA = a.acc, *accB = a.acc + (size_t)4 * a.nsys, *accC = a.acc + (size_t)8 * a.nsys;

        // ---- slot A ---------------------------------------------------------
        for_segments(a, na, list, M, [&](int sys, int64_t t0, int64_t t1) {
            const BGeo g = a.geo[sys];
            BScal *c = a.sc + sys;
            const int mode = __ldcg(&c->mode);
            if (mode == MODE_ITER) {
                const int par = __ldcg(&c->parity), restart = __ldcg(&c->restart);
                T beta, omega;
                if constexpr (sizeof(T) == 4) { beta = __ldcg(&c->beta_f); omega = __ldcg(&c->omega_f); }
                else { beta = (T)__ldcg(&c->beta); omega = (T)__ldcg(&c->omega); }
                T *p_old = (T *)(par ? a.p1 : a.p0) + g.off, *p_new = (T *)(par ? a.p0 : a.p1) + g.off;
                T *v_old = (T *)(par ? a.v1 : a.v0) + g.off, *v_new = (T *)(par ? a.v0 : a.v1) + g.off;
                DotAcc<T> dot[3];
                for (int64_t t = t0; t < t1; ++t)
                    tile_a<T, R>(g, t, tile, row + 9 * g.off, (const T *)a.r + g.off, (T *)a.rh + g.off, p_old,
                                 v_old, p_new, v_new, beta, omega, restart, dot);
                flush<T, 3>(dot, accA + (size_t)4 * sys);
            } else if (mode == MODE_UPDATE && a.mixed) {
                const bool discard = __ldcg(&c->discard) != 0;
                for (int64_t t = t0; t < t1; ++t)
                    tile_fold<T, R>(g, t, a.x64 + g.off, (T *)a.x + g.off, a.xlo ? a.xlo + g.off : nullptr,
                                    discard);
            }
        });
        if (!barrier(a, epoch, [&](int th) {
                const int *act = a.active + (size_t)list * a.nsys;
                for (int j = th; j < na; j += 256) {
                    const int sys = act[j];
                    BScal *c = a.sc + sys;
                    double *ac = accA + (size_t)4 * sys;
                    if (c->mode == MODE_ITER && !c->done) {
                        if (c->restart) {
                            c->rho = __ldcg(ac + 1);
                            c->rhat2 = __ldcg(ac + 2);
                        }
                        c->restart = 0;
                        const double alpha = c->rho / __ldcg(ac + 0);
                        if (!isfinite(alpha) || alpha == 0.0) c->done = 3;
                        else { c->alpha = alpha; publish(c); }
                    }
                    ac[0] = ac[1] = ac[2] = ac[3] = 0.0;
                }
            }))
            return;

        // ---- slot B ---------------------------------------------------------
        for_segments(a, na, list, M, [&](int sys, int64_t t0, int64_t t1) {
            const BGeo g = a.geo[sys];
            BScal *c = a.sc + sys;
            const int mode = __ldcg(&c->mode);
            if (mode == MODE_ITER && !__ldcg(&c->done)) {
                const int par = __ldcg(&c->parity);
                T alpha;
                if constexpr (sizeof(T) == 4) alpha = __ldcg(&c->alpha_f);
                else alpha = (T)__ldcg(&c->alpha);
                const T *v_new = (const T *)(par ? a.v0 : a.v1) + g.off;
                DotAcc<T> dot[3];
                for (int64_t t = t0; t < t1; ++t)
                    tile_b<T, R>(g, t, tile, row + 9 * g.off, (const T *)a.r + g.off, v_new, (T *)a.s + g.off,
                                 (T *)a.t + g.off, alpha, dot);
                flush<T, 3>(dot, accB + (size_t)4 * sys);
            } else if (mode == MODE_UPDATE) {
                DotAcc<T> rr[2];
                double d64[2] = {0.0, 0.0};
                for (int64_t t = t0; t < t1; ++t)
                    tile_true_residual<T, R>(g, t, a.row64 + 9 * g.off, a.b + g.off, a.x64 + g.off,
                                             (T *)a.r + g.off, (const T *)a.rh + g.off, rr, d64);
                flush64(d64, accB + (size_t)4 * sys);
                DotAcc<T> r1[1], r2[1];
                r1[0] = rr[0];
                r2[0] = rr[1];
                flush<T, 1>(r1, accB + (size_t)4 * sys + 3);
                flush<T, 1>(r2, accB + (size_t)4 * sys + 2);
            }
        });
        if (!barrier(a, epoch, [&](int th) {
                const int *act = a.active + (size_t)list * a.nsys;
                for (int j = th; j < na; j += 256) {
                    const int sys = act[j];
                    BScal *c = a.sc + sys;
                    double *ac = accB + (size_t)4 * sys;
                    if (c->mode == MODE_ITER && !c->done) {
                        const double ts = __ldcg(ac + 0), tt = __ldcg(ac + 1), ss = __ldcg(ac + 2);
                        if (!isfinite(ts + tt + ss)) c->done = 4;
                        else if (ss <= c->tol2) c->s_conv = 1;
                        else if (tt == 0.0) c->done = 3;
                        else { c->omega = ts / tt; publish(c); }
                    } else if (c->mode == MODE_UPDATE) {
                        const double rr64 = __ldcg(ac + 0), bb = __ldcg(ac + 1), rr = __ldcg(ac + 3);
                        const bool first = c->bb64 < 0.0;
                        c->rr64 = rr64;
                        c->bb64 = bb;
                        c->rr = rr;
                        c->tol2 = a.tol2_factor * bb;
                        c->pending = 0;
                        if (!first) c->updates += 1;
                        if (!isfinite(rr64 + bb)) c->done = 4;
                        else if (rr64 <= c->tol2) c->done = 1;
                        else if (c->max_hit) c->done = 2;
                        else {
                            c->rr_last = rr;
                            c->it_last = c->iter;
                            // residual replacement (as in the single-system
                            // solve): keep p, v and r^ and continue with beta
                            // from rho' = r^.r of the replaced residual, unless
                            // this update restarts (the first, after a dropped
                            // cycle or an ||s|| stop, or once a replaced
                            // recursion of this system has diverged)
                            const double rho_new = __ldcg(ac + 2);
                            const bool keep = a.replace && !first && !c->no_replace && !c->discard &&
                                              !c->restart && !c->s_conv && c->rho != 0.0 && c->omega != 0.0;
                            const double beta = keep ? (rho_new / c->rho) * (c->alpha / c->omega) : 0.0;
                            c->discard = 0;
                            if (keep && isfinite(beta)) {
                                c->beta = beta;
                                c->rho = rho_new;
                                publish(c);
                            } else {
                                c->restart = 1;
                                c->s_conv = 0;
                                c->alpha = c->beta = c->omega = 0.0;
                                publish(c);
                            }
                        }
                    }
                    ac[0] = ac[1] = ac[2] = ac[3] = 0.0;
                }
            }))
            return;

        // ---- slot C ---------------------------------------------------------
        for_segments(a, na, list, M, [&](int sys, int64_t t0, int64_t t1) {
            const BGeo g = a.geo[sys];
            BScal *c = a.sc + sys;
            if (__ldcg(&c->mode) == MODE_ITER && !__ldcg(&c->done)) {
                const int par = __ldcg(&c->parity), sconv = __ldcg(&c->s_conv);
                T alpha, omega;
                if constexpr (sizeof(T) == 4) { alpha = __ldcg(&c->alpha_f); omega = __ldcg(&c->omega_f); }
                else { alpha = (T)__ldcg(&c->alpha); omega = (T)__ldcg(&c->omega); }
                const T *p_new = (const T *)(par ? a.p0 : a.p1) + g.off;
                DotAcc<T> dot[2];
                for (int64_t t = t0; t < t1; ++t)
                    tile_c<T, R>(g, t, (T *)a.x + g.off, a.xlo ? a.xlo + g.off : nullptr, (T *)a.r + g.off,
                                 (const T *)a.rh + g.off, p_new,
                                 (const T *)a.s + g.off, (const T *)a.t + g.off, alpha, omega, sconv, dot);
                flush<T, 2>(dot, accC + (size_t)4 * sys);
            }
        });
        if (!barrier(a, epoch, [&](int th) {
                const int *act = a.active + (size_t)list * a.nsys;
                for (int j = th; j < na; j += 256) {
                    const int sys = act[j];
                    BScal *c = a.sc + sys;
                    double *ac = accC + (size_t)4 * sys;
                    if (c->mode == MODE_ITER && !c->done) {
                        const double rho_new = __ldcg(ac + 0), rr = __ldcg(ac + 1);
                        c->rr = rr;
                        c->iter += 1;
                        c->parity ^= 1;
                        if (!isfinite(rho_new + rr)) c->done = 4;
                        else if (c->s_conv) c->pending = 1;
                        else {
                            c->beta = (rho_new / c->rho) * (c->alpha / c->omega);
                            c->rho = rho_new;
                            publish(c);
                            if (rr <= c->tol2) c->pending = 1;
                            else if (c->iter >= c->max_iter) { c->max_hit = 1; c->pending = 1; }
                            else if (a.mixed && rr <= a.update2 * c->rr_last) c->pending = 1;
                            // MIXED guards (as in the single-system solve): a
                            // residual grown by 1e4 since the last true residual
                            // is a diverged recursion; no update for `stall`
                            // iterations forces one
                            else if (a.mixed && a.replace && !c->no_replace && rr > 1e4 * c->rr_last) {
                                // a replaced recursion that grew 100-fold has
                                // diverged: drop its correction, restart from
                                // then on
                                c->discard = 1;
                                c->no_replace = 1;
                                c->discarded += 1;
                                c->pending = 1;
                            } else if (a.mixed && rr > 1e8 * c->rr_last) c->done = 3;
                            else if (a.mixed && c->iter - c->it_last >= a.stall) c->pending = 1;
                            else if (fabs(rho_new) <= a.eps_breakdown * sqrt(c->rhat2 * rr)) {
                                c->restarts += 1;
                                if (c->restarts > 1000) c->done = 3;
                                else c->restart = 1;
                            }
                        }
                    }
                    ac[0] = ac[1] = ac[2] = ac[3] = 0.0;
                    c->mode = c->done ? MODE_SKIP : (c->pending ? MODE_UPDATE : MODE_ITER);
                }
                __syncthreads();
                rebuild_list(a, na, list);
            }))
            return;
    }
}

// b, guess and state of a solve: inner b = rhs, Dirichlet b = bnd (rscale
// 1), void b = 0; the guess takes the Dirichlet values and 0 at void DPs;
// the FP32 correction is zeroed.
__global__ void prep_kernel(int64_t N, const int8_t *__restrict__ kind, const double *__restrict__ rhs,
                            const double *__restrict__ bnd, double *__restrict__ b, double *__restrict__ p,
                            float *__restrict__ x32, float *__restrict__ x32lo) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int8_t kd = kind[k];
    double bk = 0.0;
    if (kd == KIND_INNER) bk = rhs[k];
    else if (kd == KIND_DIRICHLET) bk = bnd[k];
    b[k] = bk;
    if (kd == KIND_DIRICHLET) p[k] = bk;
    else if (kd == KIND_VOID) p[k] = 0.0;
    if (x32) x32[k] = 0.0f;
    if (x32lo) x32lo[k] = 0.0f;
}

// Scalars of every system reset to "true-residual update next", full work
// list, zero accumulators (one block).
// With `subset` (device int [nsys], may be NULL) only the systems with a
// nonzero entry run; the others are marked converged.
__global__ void init_kernel(BArgs a, int max_iter, const int *__restrict__ subset) {
    for (int i = threadIdx.x; i < a.nsys; i += blockDim.x) {
        BScal c;
        memset(&c, 0, sizeof(c));
        c.max_iter = max_iter;
        c.pending = 1;
        c.restart = 1;
        c.mode = MODE_UPDATE;
        c.bb64 = -1.0;   // marks the first update
        if (subset && !subset[i]) {
            c.done = 1;
            c.pending = 0;
            c.mode = MODE_SKIP;
        }
        a.sc[i] = c;
    }
    for (int i = threadIdx.x; i < 12 * a.nsys; i += blockDim.x) a.acc[i] = 0.0;
    __syncthreads();
    // list 0: the systems that run, with their tile prefix
    int base = 0;
    int64_t wbase = 0;
    for (int c0 = 0; c0 < a.nsys; c0 += 256) {
        const int j = c0 + threadIdx.x;
        const int keep = (j < a.nsys && (!subset || subset[j])) ? 1 : 0;
        const int64_t tiles = keep ? a.geo[j].ntiles : 0;
        int cpos, ctot;
        int64_t wpos, wtot;
        scan2(keep, tiles, cpos, wpos, ctot, wtot);
        if (keep) {
            a.active[base + cpos] = j;
            a.prefix[base + cpos] = wbase + wpos;
        }
        base += ctot;
        wbase += wtot;
    }
    if (threadIdx.x == 0) {
        a.prefix[base] = wbase;
        a.state->n_active = base;
        a.state->phase_err = 0;
        a.state->list = 0;
        a.state->M = wbase;
        a.state->sweeps = 0;
    }
}

}  // namespace batch
}  // namespace mcd

using namespace mcd;
using namespace mcd::batch;

struct mcd_batch {
    int nsys = 0;
    std::vector<mcd_mesh> meshes;
    mcd_mls_params prm{};
    std::vector<int64_t> off;     // nsys + 1
    int64_t N = 0;
    // build
    Geo *geo_d = nullptr;
    int64_t *off_d = nullptr;
    int *blk_d = nullptr;
    int build_blocks = 0;
    double *row64 = nullptr;
    float *row32 = nullptr;
    double *rscale = nullptr;
    int8_t *kind = nullptr;
    unsigned long long *bad = nullptr;
    uint16_t *off16 = nullptr;    // [N][2] bf16 DP offsets of every system (network features)
    int *spmv_err = nullptr;      // error word of the systems' SpMVs
    std::vector<mcd_stencils> views;   // system i as a stencil handle over the arrays above
    // solve
    BGeo *bgeo_d = nullptr;
    int bgeo_rows = 0;            // tiling the bgeo table holds
    double *b = nullptr;
    float *f[10] = {};            // x r rh p0 p1 v0 v1 s t (FP32), xlo (low word of the correction)
    double *d[9] = {};            // the same in FP64 (FP64 mode; x unused)
    BScal *sc = nullptr;
    BScal *h_sc = nullptr;
    double *acc = nullptr;
    int *active = nullptr;
    int64_t *prefix = nullptr;
    int *subset = nullptr;        // [nsys] systems of an FP64 finish
    BState *state = nullptr;
    BState *h_state = nullptr;
    GridBarrier *bar = nullptr;
    int bar_cap = 0;
    mcd_batch_tuning tune{2, 0};
    // graph
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;
    int glaunches = 0;
};

namespace {

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename T, int R>
const void *kernel_ptr() {
    return (const void *)bicg_batch<T, R>;
}

const void *batch_kernel(int mode, int rows) {
    const bool f = mode == MCD_MIXED;
    switch (rows) {
        case 1: return f ? kernel_ptr<float, 1>() : kernel_ptr<double, 1>();
        case 4: return f ? kernel_ptr<float, 4>() : kernel_ptr<double, 4>();
        default: return f ? kernel_ptr<float, 2>() : kernel_ptr<double, 2>();
    }
}

int max_ctas_per_sm(const void *k) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0) != cudaSuccess) return 0;
    return occ;
}

mcd_status upload_tiling(mcd_batch *bt, int rows) {
    if (bt->bgeo_d && bt->bgeo_rows == rows) return MCD_OK;
    std::vector<BGeo> h(bt->nsys);
    const int ty = 8 * rows;
    for (int i = 0; i < bt->nsys; ++i) {
        const mcd_mesh &m = bt->meshes[i];
        BGeo &g = h[i];
        g.n0 = m.n[0];
        g.n1 = m.n[1];
        g.per0 = m.periodic[0] ? 1 : 0;
        g.per1 = m.periodic[1] ? 1 : 0;
        g.N = (int64_t)m.n[0] * m.n[1];
        g.off = bt->off[i];
        g.tiles_x = (m.n[0] + 31) / 32;
        g.ntiles = g.tiles_x * ((m.n[1] + ty - 1) / ty);
    }
    if (!bt->bgeo_d) MCD_CUDA_TRY(cudaMalloc(&bt->bgeo_d, bt->nsys * sizeof(BGeo)));
    MCD_CUDA_TRY(cudaMemcpy(bt->bgeo_d, h.data(), bt->nsys * sizeof(BGeo), cudaMemcpyHostToDevice));
    bt->bgeo_rows = rows;
    return MCD_OK;
}

mcd_status ensure_solver(mcd_batch *bt, int mode) {
    const size_t N = (size_t)bt->N;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (!bt->b) {
        chk(cudaMalloc(&bt->b, N * sizeof(double)));
        chk(cudaMalloc(&bt->sc, bt->nsys * sizeof(BScal)));
        chk(cudaMallocHost(&bt->h_sc, bt->nsys * sizeof(BScal)));
        chk(cudaMalloc(&bt->acc, (size_t)12 * bt->nsys * sizeof(double)));
        chk(cudaMalloc(&bt->active, (size_t)2 * bt->nsys * sizeof(int)));
        chk(cudaMalloc(&bt->prefix, (size_t)2 * (bt->nsys + 1) * sizeof(int64_t)));
        chk(cudaMalloc(&bt->subset, (size_t)bt->nsys * sizeof(int)));
        chk(cudaMalloc(&bt->state, sizeof(BState)));
        chk(cudaMallocHost(&bt->h_state, sizeof(BState)));
    }
    if (mode == MCD_MIXED && !bt->f[0])
        for (int i = 0; i < 10; ++i) chk(cudaMalloc(&bt->f[i], N * sizeof(float)));
    if (mode == MCD_FP64 && !bt->d[1])
        for (int i = 1; i < 9; ++i) chk(cudaMalloc(&bt->d[i], N * sizeof(double)));
    const int need = 4 * device_sms();   // largest grid any tiling launches
    if (bt->bar_cap < need) {
        cudaFree(bt->bar);
        bt->bar = nullptr;
        chk(cudaMalloc(&bt->bar, barrier_bytes(need)));
        bt->bar_cap = need;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("batch solver allocation: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    return MCD_OK;
}

struct Launch {
    BArgs args;
    const void *kernel;
    int grid;
};

mcd_status make_launch(mcd_batch *bt, double *p, const mcd_solve_params *prm, Launch &L) {
    const int rows = bt->tune.rows;
    mcd_status s = upload_tiling(bt, rows);
    if (s != MCD_OK) return s;
    const void *k = batch_kernel(prm->mode, rows);
    const int occ = max_ctas_per_sm(k);
    if (occ <= 0) {
        set_error("batch kernel cannot be resident on this device");
        return MCD_ECUDA;
    }
    const int cps = std::min(bt->tune.ctas_per_sm > 0 ? bt->tune.ctas_per_sm : 4, occ);
    L.grid = std::min(cps, 4) * device_sms();
    L.kernel = k;
    BArgs &a = L.args;
    memset(&a, 0, sizeof(a));
    a.nsys = bt->nsys;
    a.geo = bt->bgeo_d;
    a.kind = bt->kind;
    a.row64 = bt->row64;
    a.b = bt->b;
    a.x64 = p;
    const bool mixed = prm->mode == MCD_MIXED;
    if (mixed) {
        a.row = bt->row32;
        a.x = bt->f[0]; a.r = bt->f[1]; a.rh = bt->f[2]; a.p0 = bt->f[3]; a.p1 = bt->f[4];
        a.v0 = bt->f[5]; a.v1 = bt->f[6]; a.s = bt->f[7]; a.t = bt->f[8];
        a.xlo = bt->f[9];
    } else {
        a.xlo = nullptr;
        a.row = bt->row64;
        a.x = p; a.r = bt->d[1]; a.rh = bt->d[2]; a.p0 = bt->d[3]; a.p1 = bt->d[4];
        a.v0 = bt->d[5]; a.v1 = bt->d[6]; a.s = bt->d[7]; a.t = bt->d[8];
    }
    a.sc = bt->sc;
    a.acc = bt->acc;
    a.active = bt->active;
    a.prefix = bt->prefix;
    a.state = bt->state;
    a.bar = bt->bar;
    a.mixed = mixed ? 1 : 0;
    a.tol2_factor = prm->tol * prm->tol;
    const double upd = (prm->inner_tol > 0.0 && prm->inner_tol < 1.0) ? prm->inner_tol : 0.3;
    a.update2 = upd * upd;
    a.replace = (mixed && prm->update_restart != 1) ? 1 : 0;
    a.stall = 1024;
    a.eps_breakdown = mixed ? 1e-12 : 1e-14;
    const long long mi = prm->max_iter > 0 ? prm->max_iter : (1 << 30);
    a.budget = (int)std::min<long long>(mi * 2 + 64, 1 << 30);
    a.spin_limit = 1ll << 21;
    return MCD_OK;
}

// The launches of one solve on `stream`: prep, init, barrier reset, the
// persistent kernel.  With `timed` the persistent launch is wrapped in a
// KTimer (direct launches); inside a graph capture it is not.
mcd_status enqueue_solve(mcd_batch *bt, const double *rhs, const double *bnd, double *p,
                         const mcd_solve_params *prm, Launch &L, cudaStream_t s, bool capture,
                         const int *subset = nullptr) {
    const int64_t N = bt->N;
    const unsigned eb = (unsigned)((N + 255) / 256);
    float *x32 = prm->mode == MCD_MIXED ? bt->f[0] : nullptr;
    float *x32lo = prm->mode == MCD_MIXED ? bt->f[9] : nullptr;
    const int max_iter = prm->max_iter > 0 ? prm->max_iter : (1 << 30);
    if (capture) {
        prep_kernel<<<eb, 256, 0, s>>>(N, bt->kind, rhs, bnd, bt->b, p, x32, x32lo);
        init_kernel<<<1, 256, 0, s>>>(L.args, max_iter, subset);
    } else {
        MCD_KLAUNCH(MCD_K_OTHER, s, prep_kernel<<<eb, 256, 0, s>>>(N, bt->kind, rhs, bnd, bt->b, p, x32, x32lo));
        MCD_KLAUNCH(MCD_K_OTHER, s, init_kernel<<<1, 256, 0, s>>>(L.args, max_iter, subset));
    }
    MCD_LAUNCH_CHECK();
    MCD_CUDA_TRY(cudaMemsetAsync(bt->bar, 0, barrier_bytes(L.grid), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&L.args};
    if (capture) {
        MCD_CUDA_TRY(cudaLaunchKernelExC(&cfg, L.kernel, args));
    } else {
        KTimer kt(MCD_K_BATCH, s);
        MCD_CUDA_TRY(cudaLaunchKernelExC(&cfg, L.kernel, args));
    }
    return MCD_OK;
}

// Continue a solve whose launch ran out of sweeps.
mcd_status continue_solve(mcd_batch *bt, Launch &L, cudaStream_t s) {
    MCD_CUDA_TRY(cudaMemsetAsync(bt->bar, 0, barrier_bytes(L.grid), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&L.args};
    KTimer kt(MCD_K_BATCH, s);
    MCD_CUDA_TRY(cudaLaunchKernelExC(&cfg, L.kernel, args));
    return MCD_OK;
}

std::string graph_key(const mcd_batch *bt, const double *rhs, const double *bnd, const double *p,
                      const mcd_solve_params *prm) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%p %p %p %d %.17g %d %.17g %d %d", (const void *)rhs, (const void *)bnd,
             (const void *)p, prm->mode, prm->tol, prm->max_iter, prm->inner_tol, bt->tune.rows,
             bt->tune.ctas_per_sm);
    return buf;
}

mcd_status run_solve(mcd_batch *bt, const double *rhs, const double *bnd, double *p,
                     const mcd_solve_params *prm, bool use_graph, cudaStream_t s, Launch &L) {
    mcd_status st = make_launch(bt, p, prm, L);
    if (st != MCD_OK) return st;
    if (use_graph) {
        const std::string key = graph_key(bt, rhs, bnd, p, prm);
        if (!bt->gexec || key != bt->gkey) {
            if (bt->gexec) {
                cudaGraphExecDestroy(bt->gexec);
                bt->gexec = nullptr;
            }
            cudaStream_t cs;
            MCD_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = enqueue_solve(bt, rhs, bnd, p, prm, L, cs, true);
                e = cudaStreamEndCapture(cs, &graph);
            }
            if (e == cudaSuccess && st == MCD_OK) e = cudaGraphInstantiate(&bt->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cs);
            if (st != MCD_OK) return st;
            if (e != cudaSuccess) {
                set_error(std::string("batch solve graph capture: ") + cudaGetErrorString(e));
                return MCD_ECUDA;
            }
            bt->gkey = key;
            bt->glaunches = 3;   // prep, init, persistent solve
        }
        count_launches(bt->glaunches);
        KTimer kt(MCD_K_BATCH, s, 0);
        MCD_CUDA_TRY(cudaGraphLaunch(bt->gexec, s));
        return MCD_OK;
    }
    return enqueue_solve(bt, rhs, bnd, p, prm, L, s, false);
}

// Wait for the solve, continue it while sweeps ran out, then fill results.
mcd_status finish_solve(mcd_batch *bt, Launch &L, mcd_batch_result *results, cudaStream_t s) {
    for (int round = 0;; ++round) {
        MCD_CUDA_TRY(cudaMemcpyAsync(bt->h_state, bt->state, sizeof(BState), cudaMemcpyDeviceToHost, s));
        MCD_CUDA_TRY(cudaStreamSynchronize(s));
        const BState &h = *bt->h_state;
        if (h.phase_err) {
            set_error("batch solve: a grid barrier timed out");
            return MCD_ETIMEOUT;
        }
        if (h.n_active == 0) break;
        if (round >= 64) {
            set_error("batch solve: launch budget exhausted");
            return MCD_ENOCONV;
        }
        mcd_status st = continue_solve(bt, L, s);
        if (st != MCD_OK) return st;
    }
    MCD_CUDA_TRY(cudaMemcpyAsync(bt->h_sc, bt->sc, bt->nsys * sizeof(BScal), cudaMemcpyDeviceToHost, s));
    MCD_CUDA_TRY(cudaStreamSynchronize(s));
    mcd_status worst = MCD_OK;
    for (int i = 0; i < bt->nsys; ++i) {
        const BScal &c = bt->h_sc[i];
        mcd_status si = MCD_ENOCONV;
        if (c.done == 1) si = MCD_OK;
        else if (c.done == 3) si = MCD_EBREAKDOWN;
        else if (c.done == 4) si = MCD_ENONFINITE;
        if (results) {
            results[i].status = si;
            results[i].iters = c.iter;
            results[i].updates = c.updates;
            results[i].rel_res = c.bb64 > 0.0 ? sqrt(c.rr64 / c.bb64) : 0.0;
            results[i].fallback = 0;
            results[i].discarded = c.discarded;
        }
        if (si != MCD_OK && worst == MCD_OK) worst = si;
    }
    if (worst != MCD_OK) set_error("batch solve: some systems did not converge (see the per-system results)");
    return worst;
}

mcd_status check_params(const mcd_batch *bt, const mcd_solve_params *prm) {
    MCD_CHECK_ARG(prm, "NULL parameters");
    MCD_CHECK_ARG(prm->tol > 0.0, "tol must be positive");
    MCD_CHECK_ARG(prm->mode == MCD_FP64 || prm->mode == MCD_MIXED, "unknown mode");
    MCD_CHECK_ARG(prm->mode != MCD_MIXED || bt->row32, "MIXED solve needs an MCD_MIXED batch");
    return MCD_OK;
}

}  // namespace

extern "C" mcd_status mcd_batch_create(const mcd_mesh *meshes, int count, const mcd_mls_params *prm,
                                       mcd_batch **out) {
    MCD_CHECK_ARG(meshes && prm && out && count > 0, "NULL argument or empty batch");
    MCD_CHECK_ARG(prm->r_e > 0.0 && prm->r_s > 0.0, "r_e and r_s must be positive");
    MCD_CHECK_ARG(prm->weight_kind == MCD_W_GAUSS || prm->weight_kind == MCD_W_COS2 ||
                      prm->weight_kind == MCD_W_LSMPS,
                  "unknown weight_kind");
    if (prm->support != 0 && prm->support != 1) {
        set_error("batched systems use the 3x3 stencil (support 1)");
        return MCD_ENOTSUP;
    }
    MCD_CHECK_ARG(prm->precision == MCD_FP64 || prm->precision == MCD_MIXED, "unknown precision");
    for (int b = 1; b < 128; ++b)
        if (prm->bc_kind[b] == MCD_BC_NEUMANN) {
            set_error("the batched solve supports Dirichlet boundary ids only");
            return MCD_ENOTSUP;
        }
    for (int i = 0; i < count; ++i) {
        const mcd_mesh &m = meshes[i];
        if (m.dim != 2) {
            set_error("the batched solve is 2D only");
            return MCD_ENOTSUP;
        }
        MCD_CHECK_ARG(m.n[0] >= 1 && m.n[1] >= 1 && m.l0 > 0.0, "bad mesh in batch");
        MCD_CHECK_ARG((int64_t)m.n[0] * m.n[1] < (1ll << 31), "mesh too large");
    }
    mcd_batch *bt = new mcd_batch();
    bt->nsys = count;
    bt->meshes.assign(meshes, meshes + count);
    bt->prm = *prm;
    bt->off.resize(count + 1);
    std::vector<Geo> geo(count);
    std::vector<int> blk(count);
    int64_t at = 0;
    int64_t blocks = 0;
    for (int i = 0; i < count; ++i) {
        bt->off[i] = at;
        geo[i] = make_geo(meshes[i]);
        at += geo[i].N;
        blk[i] = (int)blocks;
        blocks += (geo[i].N + 127) / 128;
    }
    bt->off[count] = at;
    bt->N = at;
    if (blocks >= (1ll << 31)) {
        delete bt;
        set_error("batch too large");
        return MCD_EINVAL;
    }
    bt->build_blocks = (int)blocks;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    chk(cudaMalloc(&bt->geo_d, count * sizeof(Geo)));
    chk(cudaMalloc(&bt->off_d, (count + 1) * sizeof(int64_t)));
    chk(cudaMalloc(&bt->blk_d, count * sizeof(int)));
    chk(cudaMalloc(&bt->row64, (size_t)9 * at * sizeof(double)));
    if (prm->precision == MCD_MIXED) chk(cudaMalloc(&bt->row32, (size_t)9 * at * sizeof(float)));
    chk(cudaMalloc(&bt->rscale, (size_t)at * sizeof(double)));
    chk(cudaMalloc(&bt->kind, (size_t)at));
    chk(cudaMalloc(&bt->bad, sizeof(unsigned long long)));
    chk(cudaMalloc(&bt->off16, (size_t)2 * at * sizeof(uint16_t)));
    chk(cudaMalloc(&bt->spmv_err, sizeof(int)));
    if (bt->spmv_err) chk(cudaMemset(bt->spmv_err, 0, sizeof(int)));
    if (e == cudaSuccess) chk(cudaMemcpy(bt->geo_d, geo.data(), count * sizeof(Geo), cudaMemcpyHostToDevice));
    if (e == cudaSuccess)
        chk(cudaMemcpy(bt->off_d, bt->off.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (e == cudaSuccess) chk(cudaMemcpy(bt->blk_d, blk.data(), count * sizeof(int), cudaMemcpyHostToDevice));
    if (e != cudaSuccess) {
        cudaGetLastError();
        mcd_batch_destroy(bt);
        set_error(std::string("batch allocation: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    // system i as a stencil handle over the batch's own arrays (the
    // network warm start and mcd_apply_laplacian run on it unchanged)
    bt->views.resize(count);
    for (int i = 0; i < count; ++i) {
        mcd_stencils &v = bt->views[i];
        memset(&v, 0, sizeof(v));
        const int64_t o = bt->off[i];
        v.mesh = meshes[i];
        v.prm = *prm;
        v.geo = make_geo(meshes[i]);
        v.S = 9;
        v.support = 1;
        v.shape = 2;
        v.nb = 5;
        v.has_neumann = 0;
        v.row64 = bt->row64 + 9 * o;
        v.row32 = bt->row32 ? bt->row32 + 9 * o : nullptr;
        v.rscale = bt->rscale + o;
        v.kind = bt->kind + o;
        v.off16 = bt->off16 + 2 * o;
        v.bad_dp = bt->bad;
        v.spmv_err = bt->spmv_err;
        v.ws = nullptr;
    }
    *out = bt;
    return MCD_OK;
}

extern "C" void mcd_batch_destroy(mcd_batch *bt) {
    if (!bt) return;
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    cudaFree(bt->geo_d); cudaFree(bt->off_d); cudaFree(bt->blk_d);
    cudaFree(bt->row64); cudaFree(bt->row32); cudaFree(bt->rscale); cudaFree(bt->kind); cudaFree(bt->bad);
    cudaFree(bt->off16); cudaFree(bt->spmv_err);
    cudaFree(bt->bgeo_d); cudaFree(bt->b);
    for (int i = 0; i < 9; ++i) cudaFree(bt->d[i]);
    for (int i = 0; i < 10; ++i) cudaFree(bt->f[i]);
    cudaFree(bt->sc); cudaFreeHost(bt->h_sc); cudaFree(bt->acc); cudaFree(bt->active); cudaFree(bt->prefix);
    cudaFree(bt->subset);
    cudaFree(bt->state); cudaFreeHost(bt->h_state); cudaFree(bt->bar);
    delete bt;
}

extern "C" int64_t mcd_batch_offset(const mcd_batch *bt, int i) {
    if (!bt || i < 0 || i > bt->nsys) return -1;
    return bt->off[i];
}

extern "C" mcd_status mcd_batch_build(mcd_batch *bt, const double *pos_dev, const int8_t *mask_dev,
                                      mcd_stream_t stream) {
    MCD_CHECK_ARG(bt && pos_dev && mask_dev, "NULL argument");
    MCD_CUDA_TRY(cudaMemsetAsync(bt->bad, 0xff, sizeof(unsigned long long), stream));
    BatchBuildDesc d;
    d.geo = bt->geo_d;
    d.off = bt->off_d;
    d.blk_start = bt->blk_d;
    d.nsys = bt->nsys;
    d.nblocks = bt->build_blocks;
    d.pos = pos_dev;
    d.mask = mask_dev;
    d.prm = &bt->prm;
    d.row64 = bt->row64;
    d.row32 = bt->row32;
    d.rscale = bt->rscale;
    d.kind = bt->kind;
    d.bad = bt->bad;
    MCD_CUDA_TRY(launch_build_batch(d, stream));
    for (int i = 0; i < bt->nsys; ++i)
        MCD_CUDA_TRY(cnn_store_offsets(&bt->views[i], pos_dev + 2 * bt->off[i], mask_dev + bt->off[i], stream));
    return MCD_OK;
}

extern "C" const mcd_stencils *mcd_batch_stencils(const mcd_batch *bt, int i) {
    if (!bt || i < 0 || i >= bt->nsys) return nullptr;
    return &bt->views[i];
}

extern "C" mcd_status mcd_batch_check(const mcd_batch *bt, int64_t *first_bad_dp, mcd_stream_t stream) {
    MCD_CHECK_ARG(bt, "NULL batch");
    unsigned long long bad = 0;
    MCD_CUDA_TRY(cudaMemcpyAsync(&bad, bt->bad, sizeof(bad), cudaMemcpyDeviceToHost, stream));
    MCD_CUDA_TRY(cudaStreamSynchronize(stream));
    const bool fail = bad != ~0ull;
    if (first_bad_dp) *first_bad_dp = fail ? (int64_t)bad : -1;
    if (fail) {
        set_error("singular MLS moment matrix at batch DP " + std::to_string(bad));
        return MCD_ESINGULAR;
    }
    return MCD_OK;
}

extern "C" mcd_status mcd_batch_solve(mcd_batch *bt, const double *rhs_dev, const double *bnd_dev,
                                      double *p_dev, const mcd_solve_params *prm, int use_graph,
                                      mcd_batch_result *results, mcd_stream_t stream) {
    MCD_CHECK_ARG(bt && rhs_dev && bnd_dev && p_dev, "NULL argument");
    mcd_status s = check_params(bt, prm);
    if (s != MCD_OK) return s;
    s = mcd_batch_check(bt, nullptr, stream);
    if (s != MCD_OK) return s;
    s = ensure_solver(bt, prm->mode);
    if (s != MCD_OK) return s;
    if (prm->net) {
        // the learned warm start of every system, on its assembled right-hand
        // side (the prep kernel, which the solve then runs again unchanged:
        // it touches only the Dirichlet and void entries of the guess)
        const int64_t N = bt->N;
        float *x32 = prm->mode == MCD_MIXED ? bt->f[0] : nullptr;
        float *x32lo = prm->mode == MCD_MIXED ? bt->f[9] : nullptr;
        MCD_KLAUNCH(MCD_K_OTHER, stream, prep_kernel<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(
                                             N, bt->kind, rhs_dev, bnd_dev, bt->b, p_dev, x32, x32lo));
        MCD_LAUNCH_CHECK();
        for (int i = 0; i < bt->nsys; ++i) {
            s = net_warm_start(prm->net, &bt->views[i], bt->b + bt->off[i], nullptr, p_dev + bt->off[i], nullptr,
                               stream);
            if (s != MCD_OK) return s;
        }
    }
    Launch L;
    s = run_solve(bt, rhs_dev, bnd_dev, p_dev, prm, use_graph != 0, stream, L);
    if (s != MCD_OK) return s;
    std::vector<mcd_batch_result> res(bt->nsys);
    s = finish_solve(bt, L, res.data(), stream);
    if (s == MCD_ETIMEOUT || prm->mode != MCD_MIXED || s == MCD_OK) {
        if (results) std::copy(res.begin(), res.end(), results);
        return s;
    }
    // FP64 finish of the systems whose FP32 recursion failed, from their
    // last folded iterate (the failed cycle never reached it)
    std::vector<int> sub(bt->nsys, 0);
    int nfail = 0;
    for (int i = 0; i < bt->nsys; ++i)
        if (res[i].status == MCD_EBREAKDOWN || res[i].status == MCD_ENONFINITE) {
            sub[i] = 1;
            ++nfail;
        }
    if (nfail == 0) {
        if (results) std::copy(res.begin(), res.end(), results);
        return s;
    }
    s = ensure_solver(bt, MCD_FP64);
    if (s != MCD_OK) return s;
    MCD_CUDA_TRY(cudaMemcpyAsync(bt->subset, sub.data(), bt->nsys * sizeof(int), cudaMemcpyHostToDevice, stream));
    mcd_solve_params p64 = *prm;
    p64.mode = MCD_FP64;
    Launch L64;
    s = make_launch(bt, p_dev, &p64, L64);
    if (s != MCD_OK) return s;
    s = enqueue_solve(bt, rhs_dev, bnd_dev, p_dev, &p64, L64, stream, false, bt->subset);
    if (s != MCD_OK) return s;
    std::vector<mcd_batch_result> r64(bt->nsys);
    mcd_status s64 = finish_solve(bt, L64, r64.data(), stream);
    if (s64 == MCD_ETIMEOUT) return s64;
    mcd_status worst = MCD_OK;
    for (int i = 0; i < bt->nsys; ++i) {
        if (sub[i]) {
            const int mixed_iters = res[i].iters, dropped = res[i].discarded;
            res[i] = r64[i];
            res[i].iters += mixed_iters;
            res[i].fallback = 1;
            res[i].discarded = dropped;
        }
        if (res[i].status != MCD_OK && worst == MCD_OK) worst = (mcd_status)res[i].status;
    }
    if (results) std::copy(res.begin(), res.end(), results);
    if (worst != MCD_OK) set_error("batch solve: some systems did not converge (see the per-system results)");
    return worst;
}

extern "C" mcd_status mcd_batch_set_tuning(mcd_batch *bt, const mcd_batch_tuning *t) {
    MCD_CHECK_ARG(bt && t, "NULL argument");
    MCD_CHECK_ARG(t->rows == 1 || t->rows == 2 || t->rows == 4, "rows must be 1, 2 or 4");
    MCD_CHECK_ARG(t->ctas_per_sm >= 0 && t->ctas_per_sm <= 4, "ctas_per_sm must be in [0, 4]");
    bt->tune = *t;
    return MCD_OK;
}

extern "C" mcd_status mcd_batch_get_tuning(const mcd_batch *bt, mcd_batch_tuning *t) {
    MCD_CHECK_ARG(bt && t, "NULL argument");
    *t = bt->tune;
    return MCD_OK;
}

namespace {

std::string tune_key(const mcd_batch *bt, int mode) {
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the mesh sizes
    for (const auto &m : bt->meshes)
        for (int v : {m.n[0], m.n[1], m.periodic[0], m.periodic[1]}) {
            h ^= (uint64_t)(uint32_t)v;
            h *= 1099511628211ull;
        }
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    std::string name(p.name);
    for (auto &c : name)
        if (c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s sm%d%d nsys=%d N=%lld mode=%d sizes=%016llx", name.c_str(), p.major,
             p.minor, bt->nsys, (long long)bt->N, mode, (unsigned long long)h);
    return buf;
}

}  // namespace

extern "C" mcd_status mcd_batch_autotune(mcd_batch *bt, const double *rhs_dev, const double *bnd_dev,
                                         double *p_dev, const mcd_solve_params *prm, int sweeps,
                                         const char *cache_path, double *best_ms_per_sweep,
                                         mcd_stream_t stream) {
    MCD_CHECK_ARG(bt && rhs_dev && bnd_dev && p_dev, "NULL argument");
    MCD_CHECK_ARG(sweeps > 0, "sweeps must be positive");
    mcd_status s = check_params(bt, prm);
    if (s != MCD_OK) return s;
    s = mcd_batch_check(bt, nullptr, stream);
    if (s != MCD_OK) return s;
    s = ensure_solver(bt, prm->mode);
    if (s != MCD_OK) return s;
    const std::string key = tune_key(bt, prm->mode);
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            // line: <key> | rows cps ms
            const size_t bar = line.find(" | ");
            if (bar == std::string::npos || line.substr(0, bar) != key) continue;
            std::istringstream rest(line.substr(bar + 3));
            mcd_batch_tuning t{};
            double ms = 0.0;
            if (rest >> t.rows >> t.ctas_per_sm >> ms) {
                if (mcd_batch_set_tuning(bt, &t) == MCD_OK) {
                    if (best_ms_per_sweep) *best_ms_per_sweep = ms;
                    return MCD_OK;
                }
            }
        }
    }
    // candidates: tile rows x CTAs per SM; each runs `sweeps` sweeps from the
    // same start (the prep and init kernels restore it)
    mcd_solve_params p = *prm;
    const mcd_batch_tuning saved = bt->tune;
    mcd_batch_tuning best = saved;
    double best_ms = 1e300;
    cudaEvent_t e0, e1;
    MCD_CUDA_TRY(cudaEventCreate(&e0));
    MCD_CUDA_TRY(cudaEventCreate(&e1));
    for (int rows : {1, 2, 4}) {
        const int occ = max_ctas_per_sm(batch_kernel(prm->mode, rows));
        for (int cps = 1; cps <= std::min(occ, 4); ++cps) {
            bt->tune.rows = rows;
            bt->tune.ctas_per_sm = cps;
            Launch L;
            s = make_launch(bt, p_dev, &p, L);
            if (s != MCD_OK) break;
            L.args.budget = sweeps;
            s = enqueue_solve(bt, rhs_dev, bnd_dev, p_dev, &p, L, stream, false);   // warm-up
            if (s != MCD_OK) break;
            MCD_CUDA_TRY(cudaEventRecord(e0, stream));
            s = enqueue_solve(bt, rhs_dev, bnd_dev, p_dev, &p, L, stream, false);
            if (s != MCD_OK) break;
            MCD_CUDA_TRY(cudaEventRecord(e1, stream));
            MCD_CUDA_TRY(cudaEventSynchronize(e1));
            MCD_CUDA_TRY(cudaMemcpy(bt->h_state, bt->state, sizeof(BState), cudaMemcpyDeviceToHost));
            if (bt->h_state->phase_err) {
                set_error("batch autotune: a grid barrier timed out");
                s = MCD_ETIMEOUT;
                break;
            }
            float ms = 0.0f;
            MCD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const double per = ms / (double)std::max<int64_t>(1, bt->h_state->sweeps);
            if (per < best_ms) {
                best_ms = per;
                best.rows = rows;
                best.ctas_per_sm = cps;
            }
        }
        if (s != MCD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MCD_OK) {
        bt->tune = saved;
        return s;
    }
    bt->tune = best;
    if (best_ms_per_sweep) *best_ms_per_sweep = best_ms;
    if (cache_path) {
        std::ofstream outf(cache_path, std::ios::app);
        if (outf) outf << key << " | " << best.rows << " " << best.ctas_per_sm << " " << best_ms << "\n";
    }
    return MCD_OK;
}

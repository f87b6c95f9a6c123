// Bi-CGSTAB pressure solve on the MLS PPE rows (arXiv 2404.17542, Sec. 3.3:
// the linear system of Eq. (21) is solved with Bi-CGSTAB), in two modes:
//   MCD_FP64   plain FP64 Bi-CGSTAB (the baseline);
//   MCD_MIXED  FP32 Bi-CGSTAB inner solves on the FP32 rounding of the rows,
//              wrapped in iterative refinement whose residual r = b - A x and
//              update x += d are FP64 on the FP64 rows.
//
// One Bi-CGSTAB iteration is three kernels over 2D (3D) tiles of the mesh:
//   KA  p = r + beta (p - omega v) on the tile + 1-cell halo in shared
//       memory, then v = A p, partial r^.v   -> last block: alpha
//   KB  s = r - alpha v on tile + halo, t = A s, partials t.s, t.t, s.s
//                                           -> last block: omega (or stop)
//   KC  x += alpha p + omega s, r = s - omega t, partials r^.r, r.r
//                                           -> last block: beta, convergence
// Each reduction is finished by the last block to arrive (atomic ticket),
// which sums the per-block partials in block order: deterministic results.
// Scalars live on the device; the host polls them every few iterations, and
// kernels launched after convergence return at once.
#include <cuda.h>
#include <math.h>
#include <stdio.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "krylov_common.cuh"

namespace mcd {

struct Scalars {
    double rho, alpha, omega, beta;
    double rho_prev;  // rho of the previous iteration (reliable-update beta)
    double rhat2;     // ||r^||^2 (breakdown test)
    double tol2;      // squared absolute tolerance on the recursive residual
    double rr, ss, ts, tt, rv;
    double rr64, bb64;  // last FP64 residual: ||b - A x||^2, ||b||^2
    int iter, max_iter;
    int done;         // 0 running, 1 converged, 2 max_iter, 3 breakdown, 4 nonfinite
    int restart;      // next KA sets r^ = r and p = r
    int restarts;
    int s_conv;       // ||s|| small: KC does x += alpha p and stops
    unsigned long long unknowns;  // non-void DPs of the system
    // FP32 copies of alpha, omega, beta for the FP32 kernels: a per-thread
    // double-to-float conversion would run on the FP64 pipe, which on this
    // GPU is 1/64 of the FP32 rate
    float alpha_f, omega_f, beta_f;
    // persistent solver state
    int pending;      // next step is a true-residual (reliable) update
    int max_hit;      // the recursion reached max_iter
    int parity;       // p / v ping-pong buffer of the next iteration
    int phase_err;    // a grid barrier gave up (timeout)
    double rr_last;   // recursive-precision ||r||^2 at the last true residual
    int it_last;      // iteration of the last true residual
    int diverged;     // why the recursion stopped: 1 diverged (correction dropped), 2 breakdown
                      // restarts exhausted, 3 alpha breakdown, 4 t = 0, 5 non-finite dot
    int replace;      // next CA: r was replaced by the true residual; keep p, v, r^
    int net_fresh;    // the network just corrected x64: this update continues (no exit)
    int discard;      // MIXED: the cycle's recursion diverged: drop its correction, restart
    int divergences;  // cycles dropped so far
    int updates;      // true-residual updates (persistent schedule)
    int no_replace;   // a replaced recursion diverged: restart at every later update
    // FP32 kernel: the recursion's scalars as double-float pairs (hi, lo),
    // updated on the FP32 pipe at every barrier; the doubles above are
    // refreshed from them at true-residual updates and when a launch ends
    float2 rho_d, alpha_d, omega_d, rhat2_d, tol2_d, rr_last_d, rr_d, rv_d, ts_d, tt_d, ss_d;
};

// Refresh the FP32 copies (called by the single thread that updates them).
__device__ __forceinline__ void publish(Scalars *sc) {
    sc->alpha_f = (float)sc->alpha;
    sc->omega_f = (float)sc->omega;
    sc->beta_f = (float)sc->beta;
}

template <typename T> struct ScalarOf;
template <> struct ScalarOf<double> {
    __device__ static double alpha(const Scalars *sc) { return sc->alpha; }
    __device__ static double omega(const Scalars *sc) { return sc->omega; }
    __device__ static double beta(const Scalars *sc) { return sc->beta; }
};
template <> struct ScalarOf<float> {
    __device__ static float alpha(const Scalars *sc) { return sc->alpha_f; }
    __device__ static float omega(const Scalars *sc) { return sc->omega_f; }
    __device__ static float beta(const Scalars *sc) { return sc->beta_f; }
};

struct Workspace {
    int64_t N = 0;
    int nblk = 0;        // blocks of the tiled kernels
    int nblk1 = 0;       // blocks of the 1D kernels
    double *b = nullptr, *r64 = nullptr;
    // FP64 Krylov vectors
    double *dr = nullptr, *drh = nullptr, *dp[2] = {nullptr, nullptr}, *dv[2] = {nullptr, nullptr},
           *ds = nullptr, *dt = nullptr;
    // FP32 Krylov vectors
    float *fr = nullptr, *frh = nullptr, *fp[2] = {nullptr, nullptr}, *fv[2] = {nullptr, nullptr},
          *fs = nullptr, *ft = nullptr, *fd = nullptr;
    float *fdlo = nullptr;        // low part of the double-float correction (persistent MIXED)
    float *fr1 = nullptr, *fu1 = nullptr, *fq1 = nullptr;   // one-barrier kernel: second r, u, q
    double *partials = nullptr;  // [12][max(nblk, nblk1)]
    unsigned int *counter = nullptr;
    Scalars *sc = nullptr;
    Scalars *h_sc = nullptr;     // pinned host mirror
    int pstride = 0;
    GridBarrier *bar = nullptr;  // persistent-solver grid barrier
};

void free_workspace(mcd_stencils *st) {
    Workspace *w = st->ws;
    if (!w) return;
    cudaFree(w->b); cudaFree(w->r64);
    cudaFree(w->dr); cudaFree(w->drh); cudaFree(w->dp[0]); cudaFree(w->dp[1]);
    cudaFree(w->dv[0]); cudaFree(w->dv[1]); cudaFree(w->ds); cudaFree(w->dt);
    cudaFree(w->fr); cudaFree(w->frh); cudaFree(w->fp[0]); cudaFree(w->fp[1]);
    cudaFree(w->fv[0]); cudaFree(w->fv[1]); cudaFree(w->fs); cudaFree(w->ft); cudaFree(w->fd); cudaFree(w->fdlo);
    cudaFree(w->fr1); cudaFree(w->fu1); cudaFree(w->fq1);
    cudaFree(w->partials); cudaFree(w->counter); cudaFree(w->sc); cudaFree(w->bar);
    cudaFreeHost(w->h_sc);
    delete w;
    st->ws = nullptr;
}

// One block per tile.  Each thread first issues the weight loads of its R
// DPs (independent of the tile), then the halo loads; after the barrier it
// applies the stencil from shared memory.  2D keeps all 9 x R weights in
// registers; 3D (27 per DP) loads them per DP after the barrier.

// ---- KA: p = r + beta (p_old - omega v_old); v = A p; partial r^.v -------
// On a restart p = r and the shadow residual r^ is reset to r (textbook
// choice; a random shadow vector converged more slowly on these systems), and
// r^.r and r^.r^ are reduced too so that rho = r^.r.  Neumann rows (ta.kind)
// act as identity rows.
template <int G, typename T, typename A>
__global__ void __launch_bounds__(256) bicg_ka(TileArgs ta, const T *__restrict__ row, const T *__restrict__ r,
                                               T *__restrict__ rhat, const T *__restrict__ p_old,
                                               const T *__restrict__ v_old, T *__restrict__ p_new,
                                               T *__restrict__ v_new, Scalars *sc, double *partials,
                                               int pstride, unsigned int *counter) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    __shared__ T tile[HD::H];
    if (sc->done) return;
    const T beta = ScalarOf<T>::beta(sc), omega = ScalarOf<T>::omega(sc);
    const int restart = sc->restart;
    const Geo &g = ta.g;
    const int tid = threadIdx.x;
    int x0, y0, z0;
    tile_origin<G>(ta, blockIdx.x, x0, y0, z0);
    int64_t k[TL::R];
    int lx[TL::R], ly[TL::R], lz[TL::R];
    T w[TL::R][PREF ? S : 1];
    T rh[TL::R];
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
        if (PREF) load_row<S, T>(row, g.N, k[q], w[q]);
        rh[q] = (!restart && k[q] >= 0) ? rhat[k[q]] : (T)0;
    }
    for (int h = tid; h < HD::H; h += 256) {
        const int64_t j = halo_index<G>(g, h, x0, y0, z0);
        const T rj = r[j];
        tile[h] = restart ? rj : rj + beta * (p_old[j] - omega * v_old[j]);
    }
    __syncthreads();
    DotAcc<T> dot[3];
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        if (k[q] < 0) continue;
        const T pk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
        p_new[k[q]] = pk;
        T rq = rh[q];
        if (restart) {
            rq = pk;   // pk = r[k] on a restart
            rhat[k[q]] = rq;
            dot[1].add(rq, pk);
            dot[2].add(rq, rq);
        }
        T vk;
        if (ta.kind && ta.kind[k[q]] == KIND_NEUMANN) {
            vk = pk;
        } else if (PREF) {
            vk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
        } else {
            if constexpr (S > 27) {
                vk = stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
            } else {
                T wl[S];
                load_row<S, T>(row, g.N, k[q], wl);
                vk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
            }
        }
        v_new[k[q]] = vk;
        dot[0].add(rq, vk);
    }
    dot_partials<3>(dot, partials, pstride, blockIdx.x);
    double tot[3];
    if (last_block_totals<3>(partials, pstride, gridDim.x, counter, tot) && tid == 0) {
        sc->rv = tot[0];
        if (restart) {
            sc->rho = tot[1];
            sc->rhat2 = tot[2];
        }
        sc->restart = 0;
        const double alpha = sc->rho / tot[0];
        if (!isfinite(alpha) || alpha == 0.0) { sc->done = 3; return; }
        sc->alpha = alpha;
        publish(sc);
    }
}

// ---- KB: s = r - alpha v; t = A s; partials t.s, t.t, s.s ------------------
template <int G, typename T, typename A>
__global__ void __launch_bounds__(256) bicg_kb(TileArgs ta, const T *__restrict__ row, const T *__restrict__ r,
                                               const T *__restrict__ v, T *__restrict__ s_out,
                                               T *__restrict__ t_out, Scalars *sc, double *partials,
                                               int pstride, unsigned int *counter) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    __shared__ T tile[HD::H];
    if (sc->done) return;
    const T alpha = ScalarOf<T>::alpha(sc);
    const Geo &g = ta.g;
    const int tid = threadIdx.x;
    int x0, y0, z0;
    tile_origin<G>(ta, blockIdx.x, x0, y0, z0);
    int64_t k[TL::R];
    int lx[TL::R], ly[TL::R], lz[TL::R];
    T w[TL::R][PREF ? S : 1];
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
        if (PREF) load_row<S, T>(row, g.N, k[q], w[q]);
    }
    for (int h = tid; h < HD::H; h += 256) {
        const int64_t j = halo_index<G>(g, h, x0, y0, z0);
        tile[h] = r[j] - alpha * v[j];
    }
    __syncthreads();
    DotAcc<T> dot[3];
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        if (k[q] < 0) continue;
        const T sk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
        s_out[k[q]] = sk;
        T tk;
        if (ta.kind && ta.kind[k[q]] == KIND_NEUMANN) {
            tk = sk;
        } else if (PREF) {
            tk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
        } else {
            if constexpr (S > 27) {
                tk = stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
            } else {
                T wl[S];
                load_row<S, T>(row, g.N, k[q], wl);
                tk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
            }
        }
        t_out[k[q]] = tk;
        dot[0].add(tk, sk);
        dot[1].add(tk, tk);
        dot[2].add(sk, sk);
    }
    dot_partials<3>(dot, partials, pstride, blockIdx.x);
    double tot[3];
    if (last_block_totals<3>(partials, pstride, gridDim.x, counter, tot) && tid == 0) {
        sc->ts = tot[0];
        sc->tt = tot[1];
        sc->ss = tot[2];
        if (!isfinite(tot[0] + tot[1] + tot[2])) { sc->done = 4; return; }
        if (tot[2] <= sc->tol2) { sc->s_conv = 1; return; }
        if (tot[1] == 0.0) { sc->done = 3; return; }
        sc->omega = tot[0] / tot[1];
        publish(sc);
    }
}

// ---- KC: x += alpha p + omega s; r = s - omega t; partials r^.r, r.r -------
// Each thread updates KC_VEC elements spaced by the grid size, so a warp's
// loads stay coalesced and each thread keeps KC_VEC x 5 loads in flight.
constexpr int KC_VEC = 4;

template <typename T, typename A>
__global__ void __launch_bounds__(256) bicg_kc(int64_t N, T *__restrict__ x, T *__restrict__ r,
                                               const T *__restrict__ rhat, const T *__restrict__ p,
                                               const T *__restrict__ s, const T *__restrict__ t,
                                               Scalars *sc, double *partials, int pstride,
                                               unsigned int *counter, double eps_breakdown) {
    if (sc->done) return;
    const T alpha = ScalarOf<T>::alpha(sc), omega = ScalarOf<T>::omega(sc);
    const int sconv = sc->s_conv;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    DotAcc<T> dot[2];
    T xv[KC_VEC], pv[KC_VEC], sv[KC_VEC], tv[KC_VEC], hv[KC_VEC];
#pragma unroll
    for (int u = 0; u < KC_VEC; ++u) {
        const int64_t k = k0 + u * stride;
        const bool in = k < N;
        xv[u] = in ? x[k] : (T)0;
        pv[u] = in ? p[k] : (T)0;
        sv[u] = in ? s[k] : (T)0;
        tv[u] = in ? t[k] : (T)0;
        hv[u] = in ? rhat[k] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < KC_VEC; ++u) {
        const int64_t k = k0 + u * stride;
        if (k >= N) continue;
        T rk;
        if (sconv) {
            x[k] = xv[u] + alpha * pv[u];
            rk = sv[u];
        } else {
            x[k] = xv[u] + alpha * pv[u] + omega * sv[u];
            rk = sv[u] - omega * tv[u];
        }
        r[k] = rk;
        dot[0].add(hv[u], rk);
        dot[1].add(rk, rk);
    }
    dot_partials<2>(dot, partials, pstride, blockIdx.x);
    double tot[2];
    if (last_block_totals<2>(partials, pstride, gridDim.x, counter, tot) && threadIdx.x == 0) {
        const double rho_new = tot[0], rr = tot[1];
        sc->rr = rr;
        sc->iter += 1;
        if (!isfinite(rho_new + rr)) { sc->done = 4; return; }
        if (sconv) { sc->done = 1; return; }
        sc->rho_prev = sc->rho;
        sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
        sc->rho = rho_new;
        publish(sc);
        if (rr <= sc->tol2) { sc->done = 1; return; }
        if (sc->iter >= sc->max_iter) { sc->done = 2; return; }
        if (fabs(rho_new) <= eps_breakdown * sqrt(sc->rhat2 * rr)) {
            sc->restarts += 1;
            if (sc->restarts > 1000) { sc->done = 3; return; }
            sc->restart = 1;
            sc->rho = rr;
            sc->rhat2 = rr;
            sc->beta = 0.0;
            publish(sc);
            return;
        }
    }
}

// ---- FP64 residual r = b - A x (1D; neighbours through L1) ---------------
// Its last block records ||r||^2, ||b||^2 and primes the Krylov scalars for a
// (re)start from this residual with tolerance tol2 = (tol ||b||)^2.
template <int G>
__global__ void __launch_bounds__(256) residual64(Geo g, const double *__restrict__ row, const double *__restrict__ b,
                                                  const double *__restrict__ x, double *__restrict__ r,
                                                  Scalars *sc, double *partials, int pstride,
                                                  unsigned int *counter, double tol,
                                                  const int8_t *__restrict__ excl) {
    constexpr int S = Shape<G>::S;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dot[2] = {0.0, 0.0};
    if (k < N) {
        int c[3] = {0, 0, 0};
        c[0] = (int)(k % g.n[0]);
        const int64_t rest = k / g.n[0];
        if (Shape<G>::dim == 2) c[1] = (int)rest; else { c[1] = (int)(rest % g.n[1]); c[2] = (int)(rest / g.n[1]); }
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            int o[3];
            slot_offset<G>(s, o);
            const int ox = o[0], oy = o[1], oz = o[2];
            const int gx = wrap_clamp(c[0] + ox, g.n[0], g.per[0]);
            const int gy = wrap_clamp(c[1] + oy, g.n[1], g.per[1]);
            int64_t j = (int64_t)gx + (int64_t)g.n[0] * gy;
            if (Shape<G>::dim == 3) {
                const int gz = wrap_clamp(c[2] + oz, g.n[2], g.per[2]);
                j = (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
            }
            acc += row[(int64_t)s * N + k] * x[j];
        }
        const double bk = b[k];
        const double rk = (excl && excl[k] == KIND_NEUMANN) ? 0.0 : bk - acc;
        r[k] = rk;
        dot[0] = rk * rk;
        dot[1] = bk * bk;
    }
    block_partials<2, double>(dot, partials, pstride, blockIdx.x);
    double tot[2];
    if (last_block_totals<2>(partials, pstride, gridDim.x, counter, tot) && threadIdx.x == 0) {
        sc->rr64 = tot[0];
        sc->bb64 = tot[1];
        sc->rr = tot[0];
        sc->rho = tot[0];
        sc->rhat2 = tot[0];
        sc->beta = 0.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->restart = 1;
        sc->s_conv = 0;
        publish(sc);
        sc->tol2 = tol * tol * tot[1];
        if (!isfinite(tot[0] + tot[1])) sc->done = 4;
        else sc->done = (tot[0] <= sc->tol2) ? 1 : 0;
    }
}

// Reliable update of the mixed solve (Sleijpen & van der Vorst, 1996): the
// FP32 recursive residual is replaced by the true residual
// r64 = b - A64 x64 of the FP64 iterate, r32 = (float) r64.  The search
// direction p is kept; rho = r^.r32 and beta are recomputed from the new
// residual.  `prime` (or a preceding ||s|| stop) restarts the recurrence
// instead (r^ = r, p = r).  Stops (done = 1) when ||r64|| <= tol ||b||.
template <int G>
__global__ void __launch_bounds__(256) reliable_residual(Geo g, const double *__restrict__ row,
                                                         const double *__restrict__ b,
                                                         const double *__restrict__ x,
                                                         const float *__restrict__ rhat,
                                                         float *__restrict__ r32, Scalars *sc,
                                                         double *partials, int pstride,
                                                         unsigned int *counter, double tol, int prime,
                                                         const int8_t *__restrict__ excl) {
    constexpr int S = Shape<G>::S;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dot[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < N) {
        int c[3] = {0, 0, 0};
        c[0] = (int)(k % g.n[0]);
        const int64_t rest = k / g.n[0];
        if (Shape<G>::dim == 2) c[1] = (int)rest; else { c[1] = (int)(rest % g.n[1]); c[2] = (int)(rest / g.n[1]); }
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            int o[3];
            slot_offset<G>(s, o);
            const int ox = o[0], oy = o[1], oz = o[2];
            const int gx = wrap_clamp(c[0] + ox, g.n[0], g.per[0]);
            const int gy = wrap_clamp(c[1] + oy, g.n[1], g.per[1]);
            int64_t j = (int64_t)gx + (int64_t)g.n[0] * gy;
            if (Shape<G>::dim == 3) {
                const int gz = wrap_clamp(c[2] + oz, g.n[2], g.per[2]);
                j = (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
            }
            acc += row[(int64_t)s * N + k] * x[j];
        }
        const double bk = b[k];
        const double rk = (excl && excl[k] == KIND_NEUMANN) ? 0.0 : bk - acc;
        const float rf = (float)rk;
        r32[k] = rf;
        dot[0] = rk * rk;
        dot[1] = bk * bk;
        dot[2] = (double)(rhat[k] * rf);
        dot[3] = (double)(rf * rf);
    }
    block_partials<4, double>(dot, partials, pstride, blockIdx.x);
    double tot[4];
    if (last_block_totals<4>(partials, pstride, gridDim.x, counter, tot) && threadIdx.x == 0) {
        sc->rr64 = tot[0];
        sc->bb64 = tot[1];
        sc->rr = tot[3];
        sc->tol2 = tol * tol * tot[1];
        if (!isfinite(tot[0] + tot[1])) { sc->done = 4; return; }
        if (tot[0] <= sc->tol2) { sc->done = 1; return; }
        sc->done = 0;
        if (prime == 1 || sc->s_conv || sc->restart) {
            sc->rho = tot[3];
            sc->rhat2 = tot[3];
            sc->beta = 0.0;
            sc->alpha = 1.0;
            sc->omega = 1.0;
            sc->restart = 1;
            sc->s_conv = 0;
        } else if (prime == 2) {
            // replace r only; rho and beta stay those of the recursion
        } else {
            sc->beta = (tot[2] / sc->rho_prev) * (sc->alpha / sc->omega);
            sc->rho = tot[2];
            if (!isfinite(sc->beta)) {
                sc->rho = tot[3];
                sc->rhat2 = tot[3];
                sc->beta = 0.0;
                sc->restart = 1;
            }
        }
        publish(sc);
    }
}

// x64 += d32; d32 = 0 (fold the FP32 correction into the FP64 iterate).
__global__ void fold_correction(int64_t N, double *__restrict__ x, float *__restrict__ d) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) {
        x[k] += (double)d[k];
        d[k] = 0.0f;
    }
}

// Dirichlet entries of the guess take their value (b = g there); void = 0.
// Also counts the non-void DPs (the unknowns of the solve).
__global__ void fix_guess(int64_t N, const int8_t *__restrict__ kind, const double *__restrict__ b,
                          double *__restrict__ x, Scalars *sc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int8_t kd = KIND_VOID;
    if (k < N) {
        kd = kind[k];
        if (kd == KIND_DIRICHLET) x[k] = b[k];
        else if (kd == KIND_VOID) x[k] = 0.0;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, kd != KIND_VOID);
    if ((threadIdx.x & 31) == 0 && ballot)
        atomicAdd(&sc->unknowns, (unsigned long long)__popc(ballot));
}

static mcd_status ensure_workspace(mcd_stencils *st, int mode) {
    Workspace *w = st->ws;
    const Geo &g = st->geo;
    const int64_t N = g.N;
    if (!w) {
        w = new Workspace();
        st->ws = w;
        w->N = N;
        int bx, by, bz;
        if (g.dim == 2) {
            bx = (g.n[0] + Tile<2>::X - 1) / Tile<2>::X;
            by = (g.n[1] + Tile<2>::Y - 1) / Tile<2>::Y;
            bz = 1;
        } else {
            bx = (g.n[0] + Tile<3>::X - 1) / Tile<3>::X;
            by = (g.n[1] + Tile<3>::Y - 1) / Tile<3>::Y;
            bz = (g.n[2] + Tile<3>::Z - 1) / Tile<3>::Z;
        }
        w->nblk = bx * by * bz;
        w->nblk1 = (int)((N + 255) / 256);
        w->pstride = std::max(w->nblk, w->nblk1);
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        chk(cudaMalloc(&w->b, N * sizeof(double)));
        chk(cudaMalloc(&w->r64, N * sizeof(double)));
        chk(cudaMalloc(&w->partials, 12 * (size_t)w->pstride * sizeof(double)));
        chk(cudaMalloc(&w->counter, sizeof(unsigned int)));
        chk(cudaMalloc(&w->sc, sizeof(Scalars)));
        chk(cudaMalloc(&w->bar, barrier_bytes(w->pstride)));
        chk(cudaMallocHost(&w->h_sc, sizeof(Scalars)));
        if (e == cudaSuccess) e = cudaMemset(w->counter, 0, sizeof(unsigned int));
        if (e != cudaSuccess) {
            set_error(std::string("solver workspace: ") + cudaGetErrorString(e));
            free_workspace(st);
            return MCD_ENOMEM;
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (mode == MCD_FP64 && !w->dr) {
        chk(cudaMalloc(&w->dr, N * sizeof(double)));
        chk(cudaMalloc(&w->drh, N * sizeof(double)));
        for (int i = 0; i < 2; ++i) {
            chk(cudaMalloc(&w->dp[i], N * sizeof(double)));
            chk(cudaMalloc(&w->dv[i], N * sizeof(double)));
        }
        chk(cudaMalloc(&w->ds, N * sizeof(double)));
        chk(cudaMalloc(&w->dt, N * sizeof(double)));
    }
    if (mode == MCD_MIXED && !w->fr) {
        chk(cudaMalloc(&w->fr, N * sizeof(float)));
        chk(cudaMalloc(&w->frh, N * sizeof(float)));
        for (int i = 0; i < 2; ++i) {
            chk(cudaMalloc(&w->fp[i], N * sizeof(float)));
            chk(cudaMalloc(&w->fv[i], N * sizeof(float)));
        }
        chk(cudaMalloc(&w->fs, N * sizeof(float)));
        chk(cudaMalloc(&w->ft, N * sizeof(float)));
        chk(cudaMalloc(&w->fd, N * sizeof(float)));
        chk(cudaMalloc(&w->fdlo, N * sizeof(float)));
        if (st->geo.dim == 2) {
            chk(cudaMalloc(&w->fr1, N * sizeof(float)));
            chk(cudaMalloc(&w->fu1, N * sizeof(float)));
            chk(cudaMalloc(&w->fq1, N * sizeof(float)));
        }
        if (e == cudaSuccess) e = cudaMemset(w->frh, 0, N * sizeof(float));
    }
    if (e != cudaSuccess) {
        set_error(std::string("solver vectors: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    return MCD_OK;
}

template <typename T> struct Vecs {
    T *x, *r, *rh, *p[2], *v[2], *s, *t;
};

static int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 1;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
        return v > 0 ? v : 1;
    }();
    return n;
}

template <typename K>
static int occupancy(K kernel) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, 256, 0) != cudaSuccess || blocks < 1)
        return 1;
    return blocks;
}

// Launch `count` Bi-CGSTAB iterations (3 kernels each); parity selects the
// p / v ping-pong buffers and is advanced.
template <int G, typename T, typename A>
static mcd_status launch_iters(const mcd_stencils *st, const T *row, Vecs<T> &vv, int &parity,
                               int count, double eps_breakdown, cudaStream_t stream) {
    Workspace *w = st->ws;
    const Geo &g = st->geo;
    TileArgs ta;
    ta.g = g;
    ta.bx = (g.n[0] + Tile<G>::X - 1) / Tile<G>::X;
    ta.by = (g.n[1] + Tile<G>::Y - 1) / Tile<G>::Y;
    ta.bz = (Shape<G>::dim == 3) ? (g.n[2] + Tile<G>::Z - 1) / Tile<G>::Z : 1;
    ta.ntiles = ta.bx * ta.by * ta.bz;
    ta.kind = st->has_neumann ? st->kind : nullptr;
    // one block per tile for KA / KB; KC threads take KC_VEC elements each
    const int grid_a = ta.ntiles;
    const int grid_b = ta.ntiles;
    const int grid_c = (int)std::max<int64_t>(1, (g.N + 256 * KC_VEC - 1) / (256 * KC_VEC));
    for (int it = 0; it < count; ++it) {
        const int a = parity, b = parity ^ 1;
        MCD_KLAUNCH(MCD_K_BICG_A, stream, bicg_ka<G, T, A><<<grid_a, 256, 0, stream>>>(ta, row, vv.r, vv.rh, vv.p[a], vv.v[a], vv.p[b],
                                                        vv.v[b], w->sc, w->partials, w->pstride, w->counter));
        MCD_KLAUNCH(MCD_K_BICG_B, stream, bicg_kb<G, T, A><<<grid_b, 256, 0, stream>>>(ta, row, vv.r, vv.v[b], vv.s, vv.t, w->sc,
                                                        w->partials, w->pstride, w->counter));
        MCD_KLAUNCH(MCD_K_BICG_C, stream, bicg_kc<T, A><<<grid_c, 256, 0, stream>>>(g.N, vv.x, vv.r, vv.rh, vv.p[b], vv.s, vv.t, w->sc,
                                                    w->partials, w->pstride, w->counter, eps_breakdown));
        parity = b;
    }
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

static mcd_status read_scalars(Workspace *w, cudaStream_t stream) {
    MCD_CUDA_TRY(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, stream));
    MCD_CUDA_TRY(cudaStreamSynchronize(stream));
    return MCD_OK;
}

// Run Bi-CGSTAB until the device flags `done`.  The chunk of iterations
// between host checks grows geometrically up to check_every.
template <int G, typename T, typename A>
static mcd_status run_krylov(const mcd_stencils *st, const T *row, Vecs<T> &vv, int check_every,
                             double eps_breakdown, int max_launch, cudaStream_t stream) {
    Workspace *w = st->ws;
    int parity = 0;
    int chunk = 4;
    int launched = 0;
    for (;;) {
        mcd_status s = launch_iters<G, T, A>(st, row, vv, parity, chunk, eps_breakdown, stream);
        if (s != MCD_OK) return s;
        launched += chunk;
        s = read_scalars(w, stream);
        if (s != MCD_OK) return s;
        if (w->h_sc->done) return MCD_OK;
        if (launched >= max_launch) {
            // the device never flagged an end: report instead of looping on
            set_error("Krylov loop exceeded its launch budget without a device status");
            return MCD_ENOCONV;
        }
        chunk = std::min(chunk * 2, check_every);
    }
}

// FP64 residual b - A x; with `interior` set the Neumann rows are left out
// (their residual reads 0), which is the residual of the interior block.
template <int G>
static mcd_status residual(const mcd_stencils *st, const double *x, double tol, int interior,
                           cudaStream_t stream) {
    Workspace *w = st->ws;
    const int8_t *excl = (interior && st->has_neumann) ? st->kind : nullptr;
    MCD_KLAUNCH(MCD_K_RESIDUAL, stream, residual64<G><<<w->nblk1, 256, 0, stream>>>(st->geo, st->row64, w->b, x, w->r64, w->sc, w->partials,
                                                  w->pstride, w->counter, tol, excl));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

// One Jacobi sweep on the Neumann rows: delta_k = (b_k - (A x)_k) / a_kk for
// Neumann DPs (reads x only), then x += delta.  The Neumann block is strongly
// diagonally dominant (its rows are scaled to diagonal -1/r_s^2 and couple to
// other Neumann DPs only through nearly tangential neighbours), so a few
// sweeps solve it to rounding once the interior values are final.
template <int G>
__global__ void neumann_delta(Geo g, const double *__restrict__ row, const int8_t *__restrict__ kind,
                              const double *__restrict__ b, const double *__restrict__ x,
                              double *__restrict__ delta) {
    constexpr int S = Shape<G>::S;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N || kind[k] != KIND_NEUMANN) return;
    int c[3] = {0, 0, 0};
    c[0] = (int)(k % g.n[0]);
    const int64_t rest = k / g.n[0];
    if (Shape<G>::dim == 2) c[1] = (int)rest; else { c[1] = (int)(rest % g.n[1]); c[2] = (int)(rest / g.n[1]); }
    double acc = 0.0;
    for (int s = 0; s < S; ++s) {
        int o[3];
        slot_offset<G>(s, o);
        const int gx = wrap_clamp(c[0] + o[0], g.n[0], g.per[0]);
        const int gy = wrap_clamp(c[1] + o[1], g.n[1], g.per[1]);
        int64_t j = (int64_t)gx + (int64_t)g.n[0] * gy;
        if (Shape<G>::dim == 3) {
            const int gz = wrap_clamp(c[2] + o[2], g.n[2], g.per[2]);
            j = (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
        }
        acc += row[(int64_t)s * N + k] * x[j];
    }
    delta[k] = (b[k] - acc) / row[(int64_t)(S / 2) * N + k];
}

__global__ void neumann_apply(int64_t N, const int8_t *__restrict__ kind, const double *__restrict__ delta,
                              double *__restrict__ x) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N && kind[k] == KIND_NEUMANN) x[k] += delta[k];
}

template <int G>
static mcd_status neumann_sweeps(const mcd_stencils *st, double *x, int sweeps, cudaStream_t stream) {
    Workspace *w = st->ws;
    const int64_t N = st->geo.N;
    for (int i = 0; i < sweeps; ++i) {
        MCD_KLAUNCH(MCD_K_OTHER, stream, neumann_delta<G><<<w->nblk1, 256, 0, stream>>>(st->geo, st->row64, st->kind,
                                                                                         w->b, x, w->r64));
        MCD_KLAUNCH(MCD_K_OTHER, stream, neumann_apply<<<w->nblk1, 256, 0, stream>>>(N, st->kind, w->r64, x));
    }
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

template <int G>
static mcd_status reliable_update(const mcd_stencils *st, double *x, double tol, int prime,
                                  cudaStream_t stream) {
    Workspace *w = st->ws;
    const int64_t N = st->geo.N;
    MCD_KLAUNCH(MCD_K_OTHER, stream, fold_correction<<<w->nblk1, 256, 0, stream>>>(N, x, w->fd));
    MCD_KLAUNCH(MCD_K_RESIDUAL, stream,
                reliable_residual<G><<<w->nblk1, 256, 0, stream>>>(st->geo, st->row64, w->b, x, w->frh, w->fr,
                                                                     w->sc, w->partials, w->pstride, w->counter,
                                                                     tol, prime,
                                                                     st->has_neumann ? st->kind : nullptr));
    MCD_LAUNCH_CHECK();
    return read_scalars(w, stream);
}

// Mixed solve: FP32 Bi-CGSTAB on the FP32 rows whose iterate d32 is folded
// into the FP64 solution x, with reliable updates.  At each host check the
// recursive FP32 residual is compared with the last true residual; once it
// has fallen by the factor `update` (or the recursion claims convergence),
// x += d32 and the FP64 residual b - A64 x replaces the FP32 one.  The solve
// ends when that FP64 residual meets tol.  `updates` counts the reliable
// updates after the first.
template <int G>
static mcd_status run_mixed(const mcd_stencils *st, double *x, const mcd_solve_params *prm,
                            int check_every, int max_launch, int &updates, mcd_status &result,
                            cudaStream_t stream) {
    Workspace *w = st->ws;
    const int64_t N = st->geo.N;
    const double update = prm->inner_tol;
    MCD_CUDA_TRY(cudaMemsetAsync(w->fd, 0, N * sizeof(float), stream));
    mcd_status s = reliable_update<G>(st, x, prm->tol, 1, stream);
    if (s != MCD_OK) return s;
    updates = 0;
    if (w->h_sc->done == 4) { result = MCD_ENONFINITE; return MCD_OK; }
    if (w->h_sc->done == 1) { result = MCD_OK; return MCD_OK; }
    double rr_last = w->h_sc->rr;
    Vecs<float> vv{w->fd, w->fr, w->frh, {w->fp[0], w->fp[1]}, {w->fv[0], w->fv[1]}, w->fs, w->ft};
    int parity = 0, chunk = 4, launched = 0;
    for (;;) {
        // compensated dots keep rho meaningful far below FP32 epsilon
        s = launch_iters<G, float, float>(st, st->row32, vv, parity, chunk, 1e-12, stream);
        if (s != MCD_OK) return s;
        launched += chunk;
        s = read_scalars(w, stream);
        if (s != MCD_OK) return s;
        const Scalars &h = *w->h_sc;
        if (h.done == 3) { result = MCD_EBREAKDOWN; return MCD_OK; }
        if (h.done == 4) { result = MCD_ENONFINITE; return MCD_OK; }
        const bool want = h.done == 1 || h.done == 2 || h.s_conv || h.rr <= update * update * rr_last;
        if (want) {
            const int was_max = (h.done == 2);
            s = reliable_update<G>(st, x, prm->tol,
                                     prm->update_restart == 1 ? 1 : (prm->update_restart == 2 ? 2 : 0), stream);
            if (s != MCD_OK) return s;
            ++updates;
            if (w->h_sc->done == 1) { result = MCD_OK; return MCD_OK; }
            if (w->h_sc->done == 4) { result = MCD_ENONFINITE; return MCD_OK; }
            if (was_max || w->h_sc->iter >= w->h_sc->max_iter) { result = MCD_ENOCONV; return MCD_OK; }
            rr_last = w->h_sc->rr;
            // a restarted recurrence reads p only through the restart branch,
            // so the ping-pong parity need not change
        }
        if (launched >= max_launch) {
            set_error("Krylov loop exceeded its launch budget without a device status");
            result = MCD_ENOCONV;
            return MCD_OK;
        }
        chunk = std::min(chunk * 2, check_every);
    }
}

// ===========================================================================
// Persistent solver: one cooperative launch runs Bi-CGSTAB iterations, the
// true-residual (reliable) updates and the convergence test on the device.
// Block b owns tiles [b T / G, (b + 1) T / G) for the whole launch (T tiles,
// G blocks: the grid fills every resident slot, and the tile counts of the
// blocks differ by at most one).  The reductions of an iteration are
// finished at grid barriers: each block writes its partial sums and an
// arrival flag; block 0 waits for every flag, adds the partials in block
// order (so results are deterministic), updates the scalars (on a copy in
// its shared memory in the two-barrier kernel) and releases the others
// through one word per block on a line of its own.  Every wait is bounded:
// a block that gives up records the timeout and leaves, and so do the
// others, so the launch always ends.
// ===========================================================================

struct PArgs {
    TileArgs ta;
    int grid;                // blocks of the launch
    const void *row;         // T rows of the recursion
    const double *row64;     // FP64 rows (true residual)
    const double *b;         // FP64 right-hand side
    double *x64;             // FP64 solution
    void *x, *r, *rh, *p0, *p1, *v0, *v1, *s, *t;   // T vectors (x = correction in MIXED)
    float *xlo;              // MIXED two-barrier: low part of the correction (x, xlo), else NULL
    Scalars *sc;
    double *partials;
    int pstride;
    GridBarrier *bar;
    int mixed;               // 1: fold x into x64 at every true-residual update
    int update_mode;         // 1: restart the recursion at every update
    double update2;          // MIXED: update once rr <= update2 * rr_last
    int stall;               // MIXED: update after this many iterations without one
    double tol;
    double eps_breakdown;
    int iter_budget;         // iterations this launch may run
    long long spin_limit;
    unsigned long long *trace;   // non-NULL: block 0 stamps phase times here
    int net_exit;                // MIXED with a preconditioner network: leave the launch at each
                                 // true-residual update (done = 5) for the host to apply it
    int tma_rows;                // wide stencils: rows streamed by TMA (tmap_rows)
    CUtensorMap tmap_rows;       // rows as a [S][n_y][n_x] tensor, box one tile x 9 slots
    int tma3;                    // 2D 3x3 FP32: phase operands staged by TMA (maps3)
    struct {
        CUtensorMap rows;        // [9][n_y][n_x], box 32 x 16 x 9
        CUtensorMap halo[7];     // s, t, p0, p1, v0, v1, r as [n_y][n_x], box 40 x 18
        CUtensorMap point[3];    // r^, x, xlo, box 32 x 16
    } maps3;
    // one grid barrier per iteration (bicg_persistent1; 2D 3x3 FP32 with maps3)
    int one;
    void *r1, *u0, *u1, *q0, *q1;   // second r buffer; u = A r and q~ = sigma A v, two of each
    float q_scale, q_unscale;       // sigma = 2^k close to l0^2, and 1 / sigma (exact scalings)
    struct {
        CUtensorMap rows;        // [9][n_y][n_x], box 40 x 18 x 9 from (x0 - 4, y0 - 1)
        CUtensorMap vec[10];     // r0, r1, p0, p1, v0, v1, u0, u1, q0, q1: box 40 x 20 from (x0 - 4, y0 - 2)
    } maps1;
};

static_assert(sizeof(PArgs) <= 4096, "PArgs is passed as one kernel parameter block");

__device__ __forceinline__ int tile_first(const PArgs &a, int block) {
    return (int)((int64_t)block * a.ta.ntiles / a.grid);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase timestamps of block 0 for the first 64 iterations of a launch:
// slots 0 start, 1 A done, 2 A reduced, 3 B done, 4 B reduced, 5 C done,
// 6 C reduced.  Slot 7 of iteration 0 records the launch's operand path:
// bit 0 set, bit 1 TMA-staged 3x3 tiles, bit 2 TMA row stream, bit 3 one
// barrier per iteration.
__device__ __forceinline__ void stamp(const PArgs &a, int it, int slot) {
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && it < 64) {
        a.trace[it * 8 + slot] = global_ns();
        if (it == 0 && slot == 0)
            a.trace[7] = 1ull | (a.tma3 ? 2ull : 0ull) | (a.tma_rows ? 4ull : 0ull) | (a.one ? 8ull : 0ull);
    }
}

// Per-block stamps of iteration 10: start (after the previous barrier),
// end of the first phase, and the block's SM.
__device__ __forceinline__ void stamp_block_start(const PArgs &a, int it) {
    if (a.trace && threadIdx.x == 0 && it == 10 && blockIdx.x < 2048)
        a.trace[512 + 4096 + blockIdx.x] = global_ns();
}

__device__ __forceinline__ void stamp_block(const PArgs &a, int it) {
    if (a.trace && threadIdx.x == 0 && it == 10 && blockIdx.x < 2048) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        a.trace[512 + blockIdx.x] = global_ns();
        a.trace[512 + 2048 + blockIdx.x] = smid;
    }
}

// Block 0 releases the others: one fence per storing thread (ordering the
// scalars its thread 0 wrote before the preceding __syncthreads), then plain
// strong stores of the epoch, which the waiting blocks read with acquire
// loads.  The highest blocks are released first: with more blocks than
// threads, the blocks of the second round of stores start their phase
// about 0.3 us later, and those are then blocks 1 .. grid - 257, which the
// launch places first on their SMs (measured: no change in the phase ends).
__device__ __forceinline__ void release_all(const PArgs &a, unsigned epoch) {
    const int grid = (int)gridDim.x;
    if (1 + (int)threadIdx.x >= grid) return;
    __threadfence();
    for (int b = grid - 1 - (int)threadIdx.x; b >= 1; b -= 256) st_relaxed_u32(release_word(a.bar, grid, b), epoch);
}

// Scalars of one step of the two-barrier kernel, as its block sees them.
template <typename T> struct ScalarSnap {
    int done, perr, pend, par, restart, sconv, replace, discard;
    T alpha, omega, beta;
};

template <typename T>
__device__ __forceinline__ void take_scalars(const Scalars *sc, ScalarSnap<T> &sn) {
    if (threadIdx.x == 0) {
        sn.done = vload(&sc->done);
        sn.perr = vload(&sc->phase_err);
        sn.pend = vload(&sc->pending);
        sn.par = vload(&sc->parity);
        sn.restart = vload(&sc->restart);
        sn.sconv = vload(&sc->s_conv);
        sn.replace = vload(&sc->replace);
        sn.discard = vload(&sc->discard);
        if constexpr (sizeof(T) == 4) {
            sn.alpha = vload(&sc->alpha_f);
            sn.omega = vload(&sc->omega_f);
            sn.beta = vload(&sc->beta_f);
        } else {
            sn.alpha = vload(&sc->alpha);
            sn.omega = vload(&sc->omega);
            sn.beta = vload(&sc->beta);
        }
    }
    __syncthreads();
}

// Block 0's copy of the scalars to global memory, all but the timeout word
// (any block may set that one).
__device__ __forceinline__ void store_scalars(Scalars *dst, const Scalars &src) {
    const unsigned *sw = reinterpret_cast<const unsigned *>(&src);
    unsigned *dw = reinterpret_cast<unsigned *>(dst);
    constexpr int skip = (int)(offsetof(Scalars, phase_err) / sizeof(unsigned));
    for (int i = 0; i < (int)(sizeof(Scalars) / sizeof(unsigned)); ++i)
        if (i != skip) dw[i] = sw[i];
}

// The fields take_scalars reads, from block 0's copy (the rest goes out at
// the FP64 barriers and when the launch ends).
template <typename T>
__device__ __forceinline__ void store_step_scalars(Scalars *g, const Scalars &l) {
    g->done = l.done;
    g->pending = l.pending;
    g->parity = l.parity;
    g->restart = l.restart;
    g->s_conv = l.s_conv;
    g->replace = l.replace;
    g->discard = l.discard;
    if constexpr (sizeof(T) == 4) {
        g->alpha_f = l.alpha_f;
        g->omega_f = l.omega_f;
        g->beta_f = l.beta_f;
    } else {
        g->alpha = l.alpha;
        g->omega = l.omega;
        g->beta = l.beta;
    }
}

// ---- double-float scalar arithmetic (the FP32 kernel's scalar update) -----
// One thread of block 0 updates the recursion's scalars at every barrier.
// In FP64 that chain of divisions costs about 2 us on this GPU's 1/64-rate
// FP64 pipe; the same quantities as unevaluated float pairs take a few
// dozen FP32 operations.  Products are split with fma, sums by TwoSum, and
// a quotient is q1 + (a - q1 b) / b (about 44 significant bits), enough for
// the cancellation in rho' = r^.s - omega r^.t.  The operations assume
// normalised pairs (|lo| <= ulp(hi) / 2).  The grid's totals are not: their
// low words collect the rounding errors of every partial sum, and where a
// dot product cancels (r^.r, r^.t) the low word can reach a good fraction
// of the high one; df_norm renormalises them first.
__device__ __forceinline__ DF df_norm(DF a) {
    float s, e;
    two_sum_f(a.hi, a.lo, s, e);
    return DF{s, e};
}
__device__ __forceinline__ DF df_quick(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) {
    float s, e;
    two_sum_f(a.hi, -b.hi, s, e);
    // after cancellation of the high words the low words' difference can
    // exceed s: TwoSum, not the quick form
    return df_norm(DF{s, __fadd_rn(e, __fsub_rn(a.lo, b.lo))});
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r = df_sub(a, df_mul(b, DF{q1, 0.0f}));
    return df_quick(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ float2 df_pack(DF a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ DF df_unpack(float2 a) { return DF{a.x, a.y}; }
__device__ __forceinline__ float2 df_from(double d) {
    const float h = (float)d;
    return make_float2(h, (float)(d - (double)h));
}
__device__ __forceinline__ double df_value(float2 a) { return (double)a.x + (double)a.y; }

// Grid barrier that finishes the NV-value reduction: returns false if a wait
// gave up.  Every block writes its partial sums and then its arrival flag
// (a plain release store: no atomics on a shared word).  Block 0 polls all
// flags with its 256 threads, adds the partials in block order, runs `last`
// on thread 0 with the totals, and publishes the epoch on the release word,
// which the other blocks poll.  `epoch` counts the barriers of this launch.
template <int NV, typename Acc, typename Last>
__device__ bool grid_reduce(const PArgs &a, unsigned &epoch, Acc (&d)[NV], Last last) {
    __shared__ int s_err;
    __shared__ double s_tot[NV];
    const int tid = threadIdx.x;
    ++epoch;
    unsigned long long *tb = (a.trace && epoch < 256) ? a.trace + 6656 + epoch * 8 : nullptr;
    if (tb && blockIdx.x == 0 && tid == 0) tb[0] = global_ns();
    dot_partials<NV>(d, a.partials, a.pstride, blockIdx.x);
    if (tid == 0) s_err = 0;
    __syncthreads();
    if (tb && blockIdx.x == 0 && tid == 0) tb[1] = global_ns();
    if (tid == 0) {
        const unsigned long long tarr = tb ? global_ns() : 0ull;
        st_release(&a.bar->flag[blockIdx.x], epoch);
        if (tb) atomicMax(tb + 6, tarr);
    }
    if (blockIdx.x == 0) {
        // wait for every block's flag (each thread a strided subset) and add
        // that block's partial sums as soon as its flag is seen; the fixed
        // thread -> block assignment keeps the summation order deterministic
        double acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = 0.0;
        bool ok = true;
        for (int b = tid; b < (int)gridDim.x && ok; b += 256) ok = wait_eq(&a.bar->flag[b], epoch, a.spin_limit);
        if (!ok) s_err = 1;
        else
            for (int b = tid; b < (int)gridDim.x; b += 256) {
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[q] += __ldcg(a.partials + q * a.pstride + b);
            }
        __syncthreads();
        if (tb && tid == 0) tb[2] = global_ns();
        if (s_err) {
            if (tid == 0) a.sc->phase_err = 1;
            return false;
        }
        __shared__ double red[NV][8];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
            if ((tid & 31) == 0) red[q][tid >> 5] = acc[q];
        }
        __syncthreads();
        if (tb && tid == 0) tb[3] = global_ns();
        if (tid == 0) {
            for (int q = 0; q < NV; ++q) {
                double x = 0.0;
                for (int w = 0; w < 8; ++w) x += red[q][w];
                s_tot[q] = x;
            }
            last(s_tot);
            if (tb) tb[4] = global_ns();
        }
        __syncthreads();
        release_all(a, epoch);
        if (tb && tid == 0) tb[5] = global_ns();
    } else if (tid == 0) {
        if (!wait_eq(release_word(a.bar, gridDim.x, blockIdx.x), epoch, a.spin_limit)) {
            s_err = 1;
            a.sc->phase_err = 1;
        }
        if (tb) atomicMax(tb + 7, global_ns());
    }
    __syncthreads();
    return !s_err;
}

// The barrier of the two-barrier FP32 kernel: grid_reduce with every sum
// kept as a double-float pair (the block sums, block 0's sum over the blocks
// in block order, its shuffle tree), handed to `last` as pairs.  No FP64
// instruction is on the barrier's path up to `last`: the FP64 pipe of this
// GPU runs at 1/64 of the FP32 rate, and grid_reduce's FP64 sums over the
// blocks cost about 3 us per barrier.  (Tried and slower: records that
// carry the barrier epoch next to each value, read without a separate flag,
// and a release that carries the next phase's scalars; the fences their
// relaxed accesses need cost more than the round trips they save.)
template <int NV, typename Last>
__device__ bool grid_reduce_df(const PArgs &a, unsigned &epoch, DotAcc<float> (&d)[NV], Last last) {
    __shared__ int s_err;
    __shared__ DF s_tot[NV];
    __shared__ DF s_blk[NV][8];
    __shared__ DF s_red[NV][8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int grid = (int)gridDim.x;
    float2 *pf = reinterpret_cast<float2 *>(a.partials);
    ++epoch;
    unsigned long long *tb = (a.trace && epoch < 256) ? a.trace + 6656 + epoch * 8 : nullptr;
    if (tb && blockIdx.x == 0 && tid == 0) tb[0] = global_ns();
    DF v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        v[q] = d[q].v;
        for (int o = 16; o > 0; o >>= 1) v[q] = df_add(v[q], df_shfl_down(v[q], o));
        if (lane == 0) s_blk[q][wid] = v[q];
    }
    if (tid == 0) s_err = 0;
    __syncthreads();
    if (tid < 32) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            DF x = (tid < 8) ? s_blk[q][tid] : DF{0.0f, 0.0f};
            for (int o = 4; o > 0; o >>= 1) x = df_add(x, df_shfl_down(x, o));
            if (tid == 0) pf[q * a.pstride + blockIdx.x] = make_float2(x.hi, x.lo);
        }
        if (tid == 0) {
            if (tb && blockIdx.x == 0) tb[1] = global_ns();
            const unsigned long long tarr = tb ? global_ns() : 0ull;
            st_release(&a.bar->flag[blockIdx.x], epoch);   // after this thread's partials
            if (tb) atomicMax(tb + 6, tarr);
        }
    }
    if (blockIdx.x == 0) {
        DF acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = DF{0.0f, 0.0f};
        // every flag of this thread first, then all its partial sums in one
        // round of independent loads
        bool ok = true;
        for (int b = tid; b < grid && ok; b += 256) ok = wait_eq(&a.bar->flag[b], epoch, a.spin_limit);
        if (!ok) s_err = 1;
        else
            for (int b = tid; b < grid; b += 256) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const float2 pv = __ldcg(pf + q * a.pstride + b);
                    acc[q] = df_add(acc[q], DF{pv.x, pv.y});
                }
            }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            for (int o = 16; o > 0; o >>= 1) acc[q] = df_add(acc[q], df_shfl_down(acc[q], o));
            if (lane == 0) s_red[q][wid] = acc[q];
        }
        __syncthreads();
        if (tb && tid == 0) tb[2] = tb[3] = global_ns();
        if (s_err) {
            if (tid == 0) a.sc->phase_err = 1;
            return false;
        }
        if (tid < 32) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                DF x = (tid < 8) ? s_red[q][tid] : DF{0.0f, 0.0f};
                for (int o = 4; o > 0; o >>= 1) x = df_add(x, df_shfl_down(x, o));
                if (tid == 0) s_tot[q] = x;
            }
            if (tid == 0) {
                last(s_tot);
                if (tb) tb[4] = global_ns();
            }
        }
        __syncthreads();
        release_all(a, epoch);
        if (tb && tid == 0) tb[5] = global_ns();
    } else if (tid == 0) {
        if (!wait_eq(release_word(a.bar, grid, blockIdx.x), epoch, a.spin_limit)) {
            s_err = 1;
            a.sc->phase_err = 1;
        }
        if (tb) atomicMax(tb + 7, global_ns());
    }
    __syncthreads();
    return !s_err;
}

// Phase A over the block's tiles: p = r + beta (p_old - omega v_old) (or
// p = r on a restart, with r^ = r) on tile + halo, v = A p.
// Dots: r^.v, and on a restart r^.r and r^.r^.
template <int G, typename T>
__device__ void phase_a(const PArgs &a, T *tile, const T *p_old, const T *v_old, T *p_new, T *v_new,
                        T beta, T omega, int restart, DotAcc<T> (&dot)[3]) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    constexpr int HN = (HD::H + 255) / 256;
    const Geo &g = a.ta.g;
    const T *row = (const T *)a.row;
    const T *r = (const T *)a.r;
    T *rhat = (T *)a.rh;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        T w[TL::R][PREF ? S : 1];
        T rh[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            if (PREF) load_row<S, T>(row, g.N, k[q], w[q]);
            rh[q] = (!restart && k[q] >= 0) ? __ldcg(rhat + k[q]) : (T)0;
        }
        // all halo loads of the tile are issued before any is consumed
        T hr[HN], hp[HN], hv[HN];
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            hr[u] = hp[u] = hv[u] = (T)0;
            if (h < HD::H) {
                const int64_t j = halo_index<G>(g, h, x0, y0, z0);
                hr[u] = __ldcg(r + j);
                if (!restart) {
                    hp[u] = __ldcg(p_old + j);
                    hv[u] = __ldcg(v_old + j);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            if (h < HD::H) tile[h] = restart ? hr[u] : hr[u] + beta * (hp[u] - omega * hv[u]);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const T pk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
            p_new[k[q]] = pk;
            T rq = rh[q];
            if (restart) {
                rq = pk;   // pk = r[k] on a restart
                rhat[k[q]] = rq;
                dot[1].add(rq, pk);
                dot[2].add(rq, rq);
            }
            T vk;
            if (a.ta.kind && a.ta.kind[k[q]] == KIND_NEUMANN) {
                vk = pk;
            } else if (PREF) {
                vk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
            } else {
                if constexpr (S > 27) {
                    vk = stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
                } else {
                    T wl[S];
                    load_row<S, T>(row, g.N, k[q], wl);
                    vk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
                }
            }
            v_new[k[q]] = vk;
            dot[0].add(rq, vk);
        }
        __syncthreads();
    }
}

// Phase B: s = r - alpha v (tile + halo), t = A s; dots t.s, t.t, s.s.
template <int G, typename T>
__device__ void phase_b(const PArgs &a, T *tile, const T *v, T alpha, DotAcc<T> (&dot)[3]) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    constexpr int HN = (HD::H + 255) / 256;
    const Geo &g = a.ta.g;
    const T *row = (const T *)a.row;
    const T *r = (const T *)a.r;
    T *s_out = (T *)a.s;
    T *t_out = (T *)a.t;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        T w[TL::R][PREF ? S : 1];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            if (PREF) load_row<S, T>(row, g.N, k[q], w[q]);
        }
        T hr[HN], hv[HN];
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            hr[u] = hv[u] = (T)0;
            if (h < HD::H) {
                const int64_t j = halo_index<G>(g, h, x0, y0, z0);
                hr[u] = __ldcg(r + j);
                hv[u] = __ldcg(v + j);
            }
        }
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            if (h < HD::H) tile[h] = hr[u] - alpha * hv[u];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const T sk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
            s_out[k[q]] = sk;
            T tk;
            if (a.ta.kind && a.ta.kind[k[q]] == KIND_NEUMANN) {
                tk = sk;
            } else if (PREF) {
                tk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
            } else {
                if constexpr (S > 27) {
                    tk = stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
                } else {
                    T wl[S];
                    load_row<S, T>(row, g.N, k[q], wl);
                    tk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
                }
            }
            t_out[k[q]] = tk;
            dot[0].add(tk, sk);
            dot[1].add(tk, tk);
            dot[2].add(sk, sk);
        }
        __syncthreads();
    }
}

// Phase C (the block's own DPs): x += alpha p + omega s, r = s - omega t (or
// x += alpha p, r = s after an ||s|| stop); dots r^.r, r.r.
template <int G, typename T>
__device__ void phase_c(const PArgs &a, const T *p, T alpha, T omega, int sconv, DotAcc<T> (&dot)[2]) {
    using TL = Tile<G>;
    const Geo &g = a.ta.g;
    T *x = (T *)a.x;
    T *r = (T *)a.r;
    const T *rhat = (const T *)a.rh;
    const T *s = (const T *)a.s;
    const T *t = (const T *)a.t;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
        int64_t k[TL::R];
        T xv[TL::R], pv[TL::R], sv[TL::R], tv[TL::R], hv[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            int lx, ly, lz;
            k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx, ly, lz);
            const bool in = k[q] >= 0;
            xv[q] = in ? __ldcg(x + k[q]) : (T)0;
            pv[q] = in ? __ldcg(p + k[q]) : (T)0;
            sv[q] = in ? __ldcg(s + k[q]) : (T)0;
            tv[q] = in ? __ldcg(t + k[q]) : (T)0;
            hv[q] = in ? __ldcg(rhat + k[q]) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            T rk;
            if (sconv) {
                x[k[q]] = xv[q] + alpha * pv[q];
                rk = sv[q];
            } else {
                x[k[q]] = xv[q] + alpha * pv[q] + omega * sv[q];
                rk = sv[q] - omega * tv[q];
            }
            r[k[q]] = rk;
            dot[0].add(hv[q], rk);
            dot[1].add(rk, rk);
        }
    }
}

// Fold (MIXED): x64 += x; x = 0 over the block's own DPs.
template <int G, typename T>
__device__ void phase_fold(const PArgs &a) {
    using TL = Tile<G>;
    const Geo &g = a.ta.g;
    T *x = (T *)a.x;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            int lx, ly, lz;
            const int64_t k = tile_dp<G>(g, tid, q, x0, y0, z0, lx, ly, lz);
            if (k < 0) continue;
            double add = (double)__ldcg(x + k);
            if (a.xlo) {
                add += (double)__ldcg(a.xlo + k);
                a.xlo[k] = 0.0f;
            }
            a.x64[k] += add;
            x[k] = (T)0;
        }
    }
}

// Discard (MIXED): x = 0 (and its low part) over the block's own DPs: the
// correction of a cycle whose recursion diverged is dropped, not folded.
template <int G, typename T>
__device__ void phase_discard(const PArgs &a) {
    using TL = Tile<G>;
    const Geo &g = a.ta.g;
    T *x = (T *)a.x;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            int lx, ly, lz;
            const int64_t k = tile_dp<G>(g, tid, q, x0, y0, z0, lx, ly, lz);
            if (k < 0) continue;
            x[k] = (T)0;
            if (a.xlo) a.xlo[k] = 0.0f;
        }
    }
}

// True residual r64 = b - A64 x64 (FP64 matrix form) of the block's DPs,
// stored in the recursion's precision; Neumann rows read 0 (interior block).
// Dots ||r64||^2, ||b||^2, r^.r, r.r.
template <int G, typename T>
__device__ void phase_true_residual(const PArgs &a, DotAcc<double> (&d64)[2], DotAcc<T> (&dt)[2],
                                    T *r_out = nullptr) {
    using TL = Tile<G>;
    constexpr int S = Shape<G>::S;
    const Geo &g = a.ta.g;
    T *r = r_out ? r_out : (T *)a.r;
    const T *rhat = (const T *)a.rh;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            int lx, ly, lz;
            const int64_t k = tile_dp<G>(g, tid, q, x0, y0, z0, lx, ly, lz);
            if (k < 0) continue;
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            double acc = 0.0;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                int o[3];
                slot_offset<G>(s, o);
                const int jx = wrap_clamp(gx + o[0], g.n[0], g.per[0]);
                const int jy = wrap_clamp(gy + o[1], g.n[1], g.per[1]);
                int64_t j = (int64_t)jx + (int64_t)g.n[0] * jy;
                if (Shape<G>::dim == 3) {
                    const int jz = wrap_clamp(gz + o[2], g.n[2], g.per[2]);
                    j = (int64_t)jx + (int64_t)g.n[0] * ((int64_t)jy + (int64_t)g.n[1] * jz);
                }
                acc += __ldg(a.row64 + (int64_t)s * g.N + k) * __ldcg(a.x64 + j);
            }
            const double bk = a.b[k];
            const double rk = (a.ta.kind && a.ta.kind[k] == KIND_NEUMANN) ? 0.0 : bk - acc;
            const T rt = (T)rk;
            r[k] = rt;
            d64[0].add(rk, rk);
            d64[1].add(bk, bk);
            dt[0].add(__ldcg(rhat + k), rt);
            dt[1].add(rt, rt);
        }
    }
}

// Main loop: the textbook Bi-CGSTAB iteration (rho = r^.r computed
// directly each iteration), three grid reductions per iteration.  A
// true-residual update follows recursive convergence, an ||s|| stop,
// max_iter, and (MIXED) a fall of the recursive residual by the factor
// sqrt(update2) since the last update.  update_mode 1 restarts the recursion
// after each update; update_mode 2 replaces r only and keeps rho and beta
// (the reliable update of Sleijpen and van der Vorst, 1996).
template <int G, typename T>
__global__ void __launch_bounds__(256) bicg_persistent(PArgs a) {
    using HD = HaloDims<G>;
    __shared__ T tile[HD::H];
    Scalars *sc = a.sc;
    int iters = 0;
    unsigned epoch = 0;
    for (;;) {
        if (vload(&sc->done) || vload(&sc->phase_err)) return;
        if (vload(&sc->pending)) {
            // ---- true residual (reliable) update ----------------------------
            if (a.mixed) {
                phase_fold<G, T>(a);
                DotAcc<double> none[1];
                if (!grid_reduce<1>(a, epoch, none, [&](double *) {})) return;
            }
            DotAcc<double> d64[2];
            DotAcc<T> dt[2];
            phase_true_residual<G, T>(a, d64, dt);
            DotAcc<double> all[4];
            all[0].v = d64[0].v;
            all[1].v = d64[1].v;
            if constexpr (sizeof(T) == 4) {
                all[2].v = (double)dt[0].v.hi + (double)dt[0].v.lo;
                all[3].v = (double)dt[1].v.hi + (double)dt[1].v.lo;
            } else {
                all[2].v = dt[0].v;
                all[3].v = dt[1].v;
            }
            const double tol = a.tol;
            const int mode = a.update_mode;
            if (!grid_reduce<4>(a, epoch, all, [&](double *tot) {
                    sc->rr64 = tot[0];
                    sc->bb64 = tot[1];
                    sc->rr = tot[3];
                    sc->tol2 = tol * tol * tot[1];
                    sc->pending = 0;
                    if (!isfinite(tot[0] + tot[1])) { sc->done = 4; return; }
                    if (tot[0] <= sc->tol2) { sc->done = 1; return; }
                    if (sc->max_hit) { sc->done = 2; return; }
                    sc->rr_last = tot[3];
                    sc->it_last = sc->iter;
                    if (mode == 1 || sc->restart || sc->s_conv || !sc->iter) {
                        sc->restart = 1;
                        sc->s_conv = 0;
                        sc->alpha = sc->beta = sc->omega = 0.0;
                    }
                    publish(sc);
                }))
                return;
            continue;
        }
        if (iters >= a.iter_budget) return;
        const int it = iters;
        ++iters;
        stamp(a, it, 0);
        stamp_block_start(a, it);
        const int par = vload(&sc->parity);
        T *p_old = (T *)(par ? a.p1 : a.p0), *p_new = (T *)(par ? a.p0 : a.p1);
        T *v_old = (T *)(par ? a.v1 : a.v0), *v_new = (T *)(par ? a.v0 : a.v1);
        // ---- phase A: p, v = A p, alpha ------------------------------------
        {
            const int restart = vload(&sc->restart);
            T beta, omega;
            if constexpr (sizeof(T) == 4) { beta = vload(&sc->beta_f); omega = vload(&sc->omega_f); }
            else { beta = (T)vload(&sc->beta); omega = (T)vload(&sc->omega); }
            DotAcc<T> dot[3];
            phase_a<G, T>(a, tile, p_old, v_old, p_new, v_new, beta, omega, restart, dot);
            stamp(a, it, 1);
            stamp_block(a, it);
            if (!grid_reduce<3>(a, epoch, dot, [&](double *tot) {
                    sc->rv = tot[0];
                    if (restart) {
                        sc->rho = tot[1];
                        sc->rhat2 = tot[2];
                    }
                    sc->restart = 0;
                    const double alpha = sc->rho / tot[0];
                    if (!isfinite(alpha) || alpha == 0.0) { sc->done = 3; return; }
                    sc->alpha = alpha;
                    publish(sc);
                }))
                return;
            stamp(a, it, 2);
        }
        if (vload(&sc->done)) continue;
        // ---- phase B: s, t = A s, omega ------------------------------------
        {
            T alpha;
            if constexpr (sizeof(T) == 4) alpha = vload(&sc->alpha_f);
            else alpha = (T)vload(&sc->alpha);
            DotAcc<T> dot[3];
            phase_b<G, T>(a, tile, v_new, alpha, dot);
            stamp(a, it, 3);
            if (!grid_reduce<3>(a, epoch, dot, [&](double *tot) {
                    sc->ts = tot[0];
                    sc->tt = tot[1];
                    sc->ss = tot[2];
                    if (!isfinite(tot[0] + tot[1] + tot[2])) { sc->done = 4; return; }
                    if (tot[2] <= sc->tol2) { sc->s_conv = 1; return; }
                    if (tot[1] == 0.0) { sc->done = 3; return; }
                    sc->omega = tot[0] / tot[1];
                    publish(sc);
                }))
                return;
            stamp(a, it, 4);
        }
        if (vload(&sc->done)) continue;
        // ---- phase C: x, r, beta and the tests ------------------------------
        {
            T alpha, omega;
            if constexpr (sizeof(T) == 4) { alpha = vload(&sc->alpha_f); omega = vload(&sc->omega_f); }
            else { alpha = (T)vload(&sc->alpha); omega = (T)vload(&sc->omega); }
            const int sconv = vload(&sc->s_conv);
            DotAcc<T> dot[2];
            phase_c<G, T>(a, p_new, alpha, omega, sconv, dot);
            stamp(a, it, 5);
            const double eps = a.eps_breakdown;
            const double update2 = a.update2;
            const int mixed = a.mixed;
            const int stall = a.stall;
            if (!grid_reduce<2>(a, epoch, dot, [&](double *tot) {
                    const double rho_new = tot[0], rr = tot[1];
                    sc->rr = rr;
                    sc->iter += 1;
                    sc->parity ^= 1;
                    if (!isfinite(rho_new + rr)) { sc->done = 4; return; }
                    if (sconv) { sc->pending = 1; return; }
                    sc->rho_prev = sc->rho;
                    sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
                    sc->rho = rho_new;
                    publish(sc);
                    if (rr <= sc->tol2) { sc->pending = 1; return; }
                    if (sc->iter >= sc->max_iter) { sc->max_hit = 1; sc->pending = 1; return; }
                    if (mixed && rr <= update2 * sc->rr_last) { sc->pending = 1; return; }
                    // MIXED guards: a recursion whose residual grew by 1e4
                    // since the last true residual has diverged (stop before
                    // its correction reaches x64); one that has not fallen
                    // by the update factor for `stall` iterations takes a
                    // fresh true residual and restarts
                    if (mixed && rr > 1e8 * sc->rr_last) { sc->diverged = 1; sc->done = 3; return; }
                    if (mixed && sc->iter - sc->it_last >= stall) { sc->pending = 1; return; }
                    if (fabs(rho_new) <= eps * sqrt(sc->rhat2 * rr)) {
                        sc->restarts += 1;
                        if (sc->restarts > 1000) { sc->done = 3; return; }
                        sc->restart = 1;
                    }
                }))
                return;
            stamp(a, it, 6);
        }
    }
}

// ===========================================================================
// Two-barrier schedule.  The x / r update of iteration k is fused with the
// p / v = A p phase of iteration k + 1 (phase CA), so an iteration has two
// grid reductions instead of three:
//   CA  r = s - omega t, x += alpha p + omega s (own DPs); on tile + halo
//       p' = r + beta (p - omega v) (r from the halo's s and t), v' = A p';
//       dots r^.v', r.r, r^.r             -> alpha = (r^.r) / (r^.v'), tests
//   B   s = r - alpha v', t = A s; dots t.s, t.t, s.s, r^.s, r^.t
//                                         -> omega, and beta from
//       rho' = r^.s - omega r^.t (the recurrence of r^.r for the next r)
// alpha uses the exact r^.r of phase CA; only beta uses the recurrence.
// Modes of CA: restart (p = r, r^ = r; after a true-residual update or a
// breakdown), normal, and ||s|| stop (x += alpha p, r = s, then an update).
// ===========================================================================

// ---- TMA stream of wide-stencil rows -----------------------------------
// The 81 weights of a 9x9 row come from HBM (340 MB of FP32 rows at 1024^2
// do not stay in L2).  Instead of 81 dependent-latency loads per DP, the
// tile's rows are streamed into shared memory by TMA in chunks of 9 slots
// (one row of the 9x9 window) for the whole tile, NB chunks in
// flight.  Within a phase the chunks of the block's consecutive tiles form
// one sequence i = 9 (tile - tb) + c; buffer i % NB; the rows do not change
// during a solve, so a chunk may be fetched any time ahead of its use.  A
// phase consumes every chunk it issues, so nothing is in flight at a grid
// barrier.
template <typename T> struct RowPipe {
    static constexpr int NB = (sizeof(T) == 4) ? 3 : 2;
    static constexpr int SL = 9;                        // slots per chunk
    static constexpr int TILE = 512;                    // DPs of a wide-stencil tile (64 x 8)
    static constexpr int CHUNK = SL * TILE;             // elements per chunk
    static constexpr unsigned BYTES = CHUNK * sizeof(T);
    T *buf;              // NB * CHUNK elements of dynamic shared memory, [slot][y][x]
    uint64_t *mbar;      // NB transaction barriers
    unsigned parity;     // bit b: parity of buffer b's next completion
    bool failed;
    unsigned outstanding;   // staged phases (thread 0): bit b set while buffer b has a copy in flight
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Thread 0: fetch chunk i of the phase (tile tb + i / 9, slots 9 (i % 9) ..)
// into buffer i % NB.  x0 is a multiple of the tile width (64): the
// innermost coordinate times the element size is a multiple of 16 bytes.
template <int G, typename T>
__device__ __forceinline__ void pipe_issue(const PArgs &a, const RowPipe<T> &pp, int tb, int i) {
    using RP = RowPipe<T>;
    static_assert(Shape<G>::S <= 27 || Tile<G>::X * Tile<G>::Y == RP::TILE, "a chunk holds 9 slots of one tile");
    int x0, y0, z0;
    tile_origin<G>(a.ta, tb + i / RP::SL, x0, y0, z0);
    const int b = i % RP::NB;
    const uint32_t mb = smem_addr(pp.mbar + b);
    const uint32_t dst = smem_addr(pp.buf + (size_t)b * RP::CHUNK);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the buffer
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(RP::BYTES) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(&a.tmap_rows)), "r"(x0), "r"(y0), "r"((i % RP::SL) * RP::SL),
        "r"(mb)
        : "memory");
}

// Wait (bounded) for buffer b's next completion.
template <typename T>
__device__ __forceinline__ bool pipe_wait(RowPipe<T> &pp, int b, long long limit) {
    const uint32_t mb = smem_addr(pp.mbar + b);
    const uint32_t ph = (pp.parity >> b) & 1u;
    uint32_t done = 0;
    long long polls = 0;
    while (!done) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mb), "r"(ph)
            : "memory");
        if (!done && ++polls > limit) return false;
    }
    pp.parity ^= 1u << b;
    return true;
}

// Thread 0: start the phase's chunk sequence (total chunks).
template <int G, typename T>
__device__ __forceinline__ void pipe_start(const PArgs &a, const RowPipe<T> &pp, int tb, int total) {
    if (threadIdx.x != 0 || pp.failed) return;
    for (int i = 0; i < RowPipe<T>::NB && i < total; ++i) pipe_issue<G, T>(a, pp, tb, i);
}

// (A x)_k for the thread's TL::R DPs of the tile whose first chunk is i0,
// from the shared tile of x and the streamed rows; the same arithmetic as
// stencil_apply_rows (compensated FP32 over four accumulators, or FP64),
// slots in chunk order.  Every thread of the block calls it.
template <int G, typename T>
__device__ void pipe_stencil(const PArgs &a, RowPipe<T> &pp, int tb, int i0, int total, const T *tile,
                             const int *lx, const int *ly, T *vk) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    using RP = RowPipe<T>;
    constexpr int C = HD::S / 2, NA = 4;
    float hi[TL::R][NA], lo[TL::R][NA];
    T acc[TL::R][3];
    T xk[TL::R];
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        xk[q] = tile[tile_centre<G>(lx[q], ly[q], 0)];
#pragma unroll
        for (int u = 0; u < NA; ++u) { hi[q][u] = 0.0f; lo[q][u] = 0.0f; }
#pragma unroll
        for (int u = 0; u < 3; ++u) acc[q][u] = (T)0;
    }
    for (int c = 0; c < RP::SL; ++c) {
        const int i = i0 + c, b = i % RP::NB;
        if (!pp.failed && !pipe_wait(pp, b, a.spin_limit)) {
            pp.failed = true;
            atomicExch(&a.sc->phase_err, 5);
        }
        const T *w = pp.buf + (size_t)b * RP::CHUNK;
        // slot s = 9 c + sl sits at offset (sl, c) of the 9x9 window; it
        // goes to accumulator sl % NA (a compile-time index)
#pragma unroll
        for (int sl = 0; sl < RP::SL; ++sl) {
#pragma unroll
            for (int q = 0; q < TL::R; ++q) {
                const T ws = w[(sl * TL::Y + ly[q]) * TL::X + lx[q]];
                const int h = (lx[q] + sl) + HD::HX * (ly[q] + c);
                if constexpr (sizeof(T) == 4) {
                    float p, pe;
                    if (sl == C % RP::SL && c == C / RP::SL) {
                        p = (float)ws * (float)xk[q];   // centre weight is 0 or 1: exact
                        pe = 0.0f;
                    } else {
                        const float d = __fsub_rn((float)tile[h], (float)xk[q]);
                        p = __fmul_rn((float)ws, d);
                        pe = __fmaf_rn((float)ws, d, -p);
                    }
                    float e;
                    two_sum(hi[q][sl % NA], p, hi[q][sl % NA], e);
                    lo[q][sl % NA] = __fadd_rn(lo[q][sl % NA], __fadd_rn(e, pe));
                } else {
                    acc[q][sl % 3] += ws * tile[h];
                }
            }
        }
        __syncthreads();   // every thread is done with buffer b
        if (threadIdx.x == 0 && !pp.failed && i + RP::NB < total) pipe_issue<G, T>(a, pp, tb, i + RP::NB);
    }
#pragma unroll
    for (int q = 0; q < TL::R; ++q) {
        if constexpr (sizeof(T) == 4) {
            float h01, e01, h23, e23, hs, es;
            two_sum(hi[q][0], hi[q][1], h01, e01);
            two_sum(hi[q][2], hi[q][3], h23, e23);
            two_sum(h01, h23, hs, es);
            const float lsum = __fadd_rn(__fadd_rn(__fadd_rn(lo[q][0], lo[q][1]), __fadd_rn(lo[q][2], lo[q][3])),
                                         __fadd_rn(__fadd_rn(e01, e23), es));
            vk[q] = (T)__fadd_rn(hs, lsum);
        } else {
            vk[q] = (acc[q][0] + acc[q][1]) + acc[q][2];
        }
    }
}

// The correction of a MIXED solve as a double-float pair (x, xlo):
// x + xlo + alpha p + omega s with both products split exactly (fma) and
// the sums by TwoSum, renormalised so |xlo| <= ulp(x) / 2.  A rounding
// error e in the correction moves the true residual by A e, amplified by
// the condition number of A (1e5-1e6 on these meshes); kept in one FP32
// word the correction would separate the true residual from the recursive
// one by ~1e-2 of the residual at the last update, which is what limits how
// far an FP32 cycle can run and whether a replaced residual keeps the
// recursion going.
__device__ __forceinline__ void add_correction(float *xlo, float *x, int64_t k, float xh, float xl, float alpha,
                                               float p, float omega, float s) {
    DF acc{xh, xl};
    df_add_prod(acc, alpha, p);
    df_add_prod(acc, omega, s);
    float hi, lo;
    two_sum_f(acc.hi, acc.lo, hi, lo);
    x[k] = hi;
    xlo[k] = lo;
}

// CA_REPLACE: r already holds the true residual that replaced the recursive
// one (reliable update with residual replacement); x and r are not updated,
// p = r + beta (p_old - omega v_old) continues the recursion.
enum { CA_NORMAL = 0, CA_RESTART = 1, CA_SCONV = 2, CA_REPLACE = 3 };

template <int G, typename T>
__device__ void phase_ca(const PArgs &a, T *tile, const T *p_old, const T *v_old, T *p_new, T *v_new,
                         T alpha, T omega, T beta, int mode, DotAcc<T> (&dot)[3], RowPipe<T> &pp) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    constexpr int HN = (HD::H + 255) / 256;
    const Geo &g = a.ta.g;
    const T *row = (const T *)a.row;
    T *x = (T *)a.x;
    T *r = (T *)a.r;
    T *rhat = (T *)a.rh;
    const T *s = (const T *)a.s;
    const T *t = (const T *)a.t;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    const bool tma = (S > 27) && a.tma_rows && mode != CA_SCONV;
    const bool rep = mode == CA_REPLACE;
    const int total = RowPipe<T>::SL * (te - tb);
    if (tma) pipe_start<G, T>(a, pp, tb, total);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        T w[TL::R][PREF ? S : 1];
        T rh[TL::R], xo[TL::R], po[TL::R], so[TL::R], to[TL::R];
        float xl[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            const bool in = k[q] >= 0;
            if (PREF && mode != CA_SCONV) load_row<S, T>(row, g.N, k[q], w[q]);
            rh[q] = (mode != CA_RESTART && in) ? __ldcg(rhat + k[q]) : (T)0;
            xo[q] = (mode != CA_RESTART && !rep && in) ? __ldcg(x + k[q]) : (T)0;
            xl[q] = (a.xlo && mode != CA_RESTART && !rep && in) ? __ldcg(a.xlo + k[q]) : 0.0f;
            po[q] = (mode != CA_RESTART && !rep && in) ? __ldcg(p_old + k[q]) : (T)0;
            so[q] = (mode != CA_RESTART && in) ? __ldcg((rep ? (const T *)r : s) + k[q]) : (T)0;
            to[q] = (mode == CA_NORMAL && in) ? __ldcg(t + k[q]) : (T)0;
        }
        if (mode == CA_SCONV) {
            // x += alpha p, r = s; a true-residual update follows
#pragma unroll
            for (int q = 0; q < TL::R; ++q) {
                if (k[q] < 0) continue;
                if (a.xlo) {
                    if constexpr (sizeof(T) == 4) add_correction(a.xlo, x, k[q], xo[q], xl[q], alpha, po[q], 0.0f, 0.0f);
                } else {
                    x[k[q]] = xo[q] + alpha * po[q];
                }
                r[k[q]] = so[q];
                dot[1].add(so[q], so[q]);
                dot[2].add(rh[q], so[q]);
            }
            continue;
        }
        // p' on tile + halo (all halo loads issued before any is consumed)
        T h1[HN], h2[HN], h3[HN], h4[HN];
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            h1[u] = h2[u] = h3[u] = h4[u] = (T)0;
            if (h < HD::H) {
                const int64_t j = halo_index<G>(g, h, x0, y0, z0);
                if (mode == CA_RESTART) {
                    h1[u] = __ldcg(r + j);
                } else {
                    // CA_REPLACE: r_j = r[j] (h2 = 0 makes r_j = h1 exactly)
                    h1[u] = __ldcg((rep ? (const T *)r : s) + j);
                    if (!rep) h2[u] = __ldcg(t + j);
                    h3[u] = __ldcg(p_old + j);
                    h4[u] = __ldcg(v_old + j);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            if (h < HD::H) {
                if (mode == CA_RESTART) {
                    tile[h] = h1[u];
                } else {
                    const T rj = h1[u] - omega * h2[u];
                    tile[h] = rj + beta * (h3[u] - omega * h4[u]);
                }
            }
        }
        __syncthreads();
        T vks[TL::R];
        if (tma) pipe_stencil<G, T>(a, pp, tb, RowPipe<T>::SL * (tl - tb), total, tile, lx, ly, vks);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const T pk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
            T rk, rq = rh[q];
            if (mode == CA_RESTART) {
                rk = pk;   // p = r on a restart
                rq = pk;
                rhat[k[q]] = pk;
            } else if (rep) {
                rk = so[q];   // the replaced residual, already stored
            } else {
                rk = so[q] - omega * to[q];
                if (a.xlo) {
                    if constexpr (sizeof(T) == 4) add_correction(a.xlo, x, k[q], xo[q], xl[q], alpha, po[q], omega, so[q]);
                } else {
                    x[k[q]] = xo[q] + alpha * po[q] + omega * so[q];
                }
                r[k[q]] = rk;
            }
            p_new[k[q]] = pk;
            T vk;
            if (a.ta.kind && a.ta.kind[k[q]] == KIND_NEUMANN) {
                vk = pk;
            } else if (PREF) {
                vk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
            } else {
                if constexpr (S > 27) {
                    vk = tma ? vks[q] : stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
                } else {
                    T wl[S];
                    load_row<S, T>(row, g.N, k[q], wl);
                    vk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
                }
            }
            v_new[k[q]] = vk;
            dot[0].add(rq, vk);
            dot[1].add(rk, rk);
            dot[2].add(rq, rk);
        }
        __syncthreads();
    }
}

// Phase B of the two-barrier schedule: s = r - alpha v, t = A s; dots t.s,
// t.t, s.s, r^.s, r^.t.
template <int G, typename T>
__device__ void phase_b2(const PArgs &a, T *tile, const T *v, T alpha, DotAcc<T> (&dot)[5], RowPipe<T> &pp) {
    using HD = HaloDims<G>;
    using TL = Tile<G>;
    constexpr int S = HD::S;
    constexpr bool PREF = (S == 9);
    constexpr int HN = (HD::H + 255) / 256;
    const Geo &g = a.ta.g;
    const T *row = (const T *)a.row;
    const T *r = (const T *)a.r;
    const T *rhat = (const T *)a.rh;
    T *s_out = (T *)a.s;
    T *t_out = (T *)a.t;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    const bool tma = (S > 27) && a.tma_rows;
    const int total = RowPipe<T>::SL * (te - tb);
    if (tma) pipe_start<G, T>(a, pp, tb, total);
    for (int tl = tb; tl < te; ++tl) {
        int x0, y0, z0;
        tile_origin<G>(a.ta, tl, x0, y0, z0);
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        T w[TL::R][PREF ? S : 1];
        T rh[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<G>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            if (PREF) load_row<S, T>(row, g.N, k[q], w[q]);
            rh[q] = (k[q] >= 0) ? __ldcg(rhat + k[q]) : (T)0;
        }
        T hr[HN], hv[HN];
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            hr[u] = hv[u] = (T)0;
            if (h < HD::H) {
                const int64_t j = halo_index<G>(g, h, x0, y0, z0);
                hr[u] = __ldcg(r + j);
                hv[u] = __ldcg(v + j);
            }
        }
#pragma unroll
        for (int u = 0; u < HN; ++u) {
            const int h = tid + u * 256;
            if (h < HD::H) tile[h] = hr[u] - alpha * hv[u];
        }
        __syncthreads();
        T vks[TL::R];
        if (tma) pipe_stencil<G, T>(a, pp, tb, RowPipe<T>::SL * (tl - tb), total, tile, lx, ly, vks);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const T sk = tile[tile_centre<G>(lx[q], ly[q], lz[q])];
            s_out[k[q]] = sk;
            T tk;
            if (a.ta.kind && a.ta.kind[k[q]] == KIND_NEUMANN) {
                tk = sk;
            } else if (PREF) {
                tk = stencil_apply<G, T, (G != 2)>(w[q], tile, lx[q], ly[q], lz[q]);
            } else {
                if constexpr (S > 27) {
                    tk = tma ? vks[q] : stencil_apply_rows<G, T>(row, g.N, k[q], tile, lx[q], ly[q], lz[q]);
                } else {
                    T wl[S];
                    load_row<S, T>(row, g.N, k[q], wl);
                    tk = stencil_apply<G, T, (G != 2)>(wl, tile, lx[q], ly[q], lz[q]);
                }
            }
            t_out[k[q]] = tk;
            dot[0].add(tk, sk);
            dot[1].add(tk, tk);
            dot[2].add(sk, sk);
            dot[3].add(rh[q], sk);
            dot[4].add(rh[q], tk);
        }
        __syncthreads();
    }
}

// ---- TMA-staged phases of the two-barrier kernel (2D 3x3, FP32) ----------
// A block's phase walks its tiles with two stages in flight: while all
// threads work on tile i from shared memory, thread 0 has tile i + 1's
// operands on the way.  A stage holds everything the tile's phase reads: the
// nine weight slots of its 32 x 16 DPs (one 3D copy of the rows), 40 x 18
// halo boxes of the vectors the stencil is applied to (x from x0 - 4 so that
// each copy starts on a 16-byte boundary, y from y0 - 1), and 32 x 16 boxes
// of the point vectors.  Copies past the mesh fill zeros: on a non-periodic
// mesh those neighbours carry zero weight, and every value formed there is
// finite.  The arithmetic per DP is that of phase_ca / phase_b2.
struct Stage3 {
    static constexpr int TX = 32, TY = 16, HXB = 40, HYB = 18;
    static constexpr unsigned W_BYTES = 9u * TX * TY * 4u;      // 18432
    static constexpr unsigned H_BYTES = HXB * HYB * 4u;         // 2880
    static constexpr unsigned H_PAD = 2944u;                    // 128-byte multiple
    static constexpr unsigned P_BYTES = TX * TY * 4u;           // 2048
    static constexpr unsigned CA_TX = W_BYTES + 4u * H_BYTES + 3u * P_BYTES;
    static constexpr unsigned B_TX = W_BYTES + 2u * H_BYTES + P_BYTES;
    static constexpr unsigned BYTES = W_BYTES + 4u * H_PAD + 3u * P_BYTES;
    static constexpr int NB = 2;
    static constexpr unsigned halo_off(int q) { return W_BYTES + (unsigned)q * H_PAD; }
    static constexpr unsigned point_off(int q) { return W_BYTES + 4u * H_PAD + (unsigned)q * P_BYTES; }
};
static_assert(Tile<2>::X == Stage3::TX && Tile<2>::Y == Stage3::TY, "stage boxes are one 2D tile");
enum { H_S = 0, H_T = 1, H_P0 = 2, H_P1 = 3, H_V0 = 4, H_V1 = 5, H_R = 6 };
enum { PT_RH = 0, PT_X = 1, PT_XLO = 2 };

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mb) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mb)
        : "memory");
}

// Thread 0: tile `tl` of a phase into stage buffer b.  ca: phase CA (halos
// s, t, p_old, v_old; points r^, x, xlo), else phase B (halos r, v; point
// r^).  par: the p / v buffer the phase reads (p_old, v_old in CA; v in B).
__device__ __forceinline__ void stage_issue(const PArgs &a, RowPipe<float> &pp, int b, int tl, bool ca,
                                            int par) {
    pp.outstanding |= 1u << b;
    int x0, y0, z0;
    tile_origin<2>(a.ta, tl, x0, y0, z0);
    const uint32_t mb = smem_addr(pp.mbar + b);
    const uint32_t dst = smem_addr(pp.buf) + (uint32_t)b * Stage3::BYTES;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the buffer
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                 "r"(ca ? Stage3::CA_TX : Stage3::B_TX)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(&a.maps3.rows)), "r"(x0), "r"(y0), "r"(0), "r"(mb)
        : "memory");
    const int hx = x0 - 4, hy = y0 - 1;
    if (ca) {
        tma_2d(dst + Stage3::halo_off(0), &a.maps3.halo[H_S], hx, hy, mb);
        tma_2d(dst + Stage3::halo_off(1), &a.maps3.halo[H_T], hx, hy, mb);
        tma_2d(dst + Stage3::halo_off(2), &a.maps3.halo[par ? H_P1 : H_P0], hx, hy, mb);
        tma_2d(dst + Stage3::halo_off(3), &a.maps3.halo[par ? H_V1 : H_V0], hx, hy, mb);
        tma_2d(dst + Stage3::point_off(0), &a.maps3.point[PT_RH], x0, y0, mb);
        tma_2d(dst + Stage3::point_off(1), &a.maps3.point[PT_X], x0, y0, mb);
        tma_2d(dst + Stage3::point_off(2), &a.maps3.point[PT_XLO], x0, y0, mb);
    } else {
        tma_2d(dst + Stage3::halo_off(0), &a.maps3.halo[H_R], hx, hy, mb);
        tma_2d(dst + Stage3::halo_off(1), &a.maps3.halo[par ? H_V1 : H_V0], hx, hy, mb);
        tma_2d(dst + Stage3::point_off(0), &a.maps3.point[PT_RH], x0, y0, mb);
    }
}

// Wait (bounded) for stage b; a timeout raises the solve's error word and
// the phase runs on (its results are discarded with the launch).
__device__ __forceinline__ void stage_wait(const PArgs &a, RowPipe<float> &pp, int b) {
    if (pp.failed) return;
    if (pipe_wait(pp, b, a.spin_limit)) {
        pp.outstanding &= ~(1u << b);
    } else {
        pp.failed = true;
        atomicExch(&a.sc->phase_err, 5);
    }
}

// After a timeout: thread 0 waits (bounded) for the copies it still has in
// flight, so that none lands in shared memory the block no longer owns.
__device__ __forceinline__ void stage_drain(const PArgs &a, RowPipe<float> &pp) {
    if (threadIdx.x != 0 || !pp.failed) return;
    for (int b = 0; b < Stage3::NB; ++b)
        if (pp.outstanding & (1u << b)) {
            pipe_wait(pp, b, a.spin_limit);
            pp.outstanding &= ~(1u << b);
        }
}

// Phase CA (normal iterations) from staged operands: x, r of the last
// iteration; p = r + beta (p_old - omega v_old) on tile + halo; v = A p.
__device__ void phase_ca_staged(const PArgs &a, float *tile0, float *tile1, int par, float alpha, float omega,
                                float beta, DotAcc<float> (&dot)[3], RowPipe<float> &pp) {
    using HD = HaloDims<2>;
    using TL = Tile<2>;
    const Geo &g = a.ta.g;
    float *x = (float *)a.x;
    float *r = (float *)a.r;
    float *p_new = (float *)(par ? a.p0 : a.p1);
    float *v_new = (float *)(par ? a.v0 : a.v1);
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    const int total = te - tb;
    if (tid == 0 && !pp.failed)
        for (int i = 0; i < Stage3::NB && i < total; ++i) stage_issue(a, pp, i, tb + i, true, par);
    // Consecutive tiles build their halo tiles in alternate buffers: a thread
    // that fills tile i + 1's halo has passed no barrier since it read tile
    // i's, but every thread reading buffer (i & 1) in tile i finished before
    // the barrier of tile i + 1, which any thread passes before it refills
    // that buffer in tile i + 2.  One __syncthreads per tile.
    for (int i = 0; i < total; ++i) {
        const int b = i % Stage3::NB;
        float *tile = (i & 1) ? tile1 : tile0;
        stage_wait(a, pp, b);
        const unsigned char *st = reinterpret_cast<const unsigned char *>(pp.buf) + (size_t)b * Stage3::BYTES;
        const float *W = reinterpret_cast<const float *>(st);
        const float *S = reinterpret_cast<const float *>(st + Stage3::halo_off(0));
        const float *T = reinterpret_cast<const float *>(st + Stage3::halo_off(1));
        const float *PO = reinterpret_cast<const float *>(st + Stage3::halo_off(2));
        const float *VO = reinterpret_cast<const float *>(st + Stage3::halo_off(3));
        const float *RH = reinterpret_cast<const float *>(st + Stage3::point_off(0));
        const float *X = reinterpret_cast<const float *>(st + Stage3::point_off(1));
        const float *XL = reinterpret_cast<const float *>(st + Stage3::point_off(2));
        int x0, y0, z0;
        tile_origin<2>(a.ta, tb + i, x0, y0, z0);
        // the DPs' roles first: these are the phase's only global loads, and
        // issued here their latency overlaps the halo fill below
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        bool neu[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<2>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            neu[q] = a.ta.kind && k[q] >= 0 && __ldg(a.ta.kind + k[q]) == KIND_NEUMANN;
        }
        for (int h = tid; h < HD::H; h += 256) {
            const int hy = h / HD::HX, hx = h - hy * HD::HX;
            const int hi = hy * Stage3::HXB + hx + 3;
            const float rj = S[hi] - omega * T[hi];
            tile[h] = rj + beta * (PO[hi] - omega * VO[hi]);
        }
        float w[TL::R][9], so[TL::R], to[TL::R], po[TL::R], rh[TL::R], xo[TL::R], xl[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            const int pi = ly[q] * Stage3::TX + lx[q];
            const int hc = (ly[q] + 1) * Stage3::HXB + lx[q] + 4;
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) w[q][sl] = W[sl * (Stage3::TX * Stage3::TY) + pi];
            so[q] = S[hc]; to[q] = T[hc]; po[q] = PO[hc];
            rh[q] = RH[pi]; xo[q] = X[pi]; xl[q] = XL[pi];
        }
        __syncthreads();   // the halo tile is complete and stage b is read: refill it
        if (tid == 0 && !pp.failed && i + Stage3::NB < total) stage_issue(a, pp, b, tb + i + Stage3::NB, true, par);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const float pk = tile[tile_centre<2>(lx[q], ly[q], 0)];
            const float rk = so[q] - omega * to[q];
            add_correction(a.xlo, x, k[q], xo[q], xl[q], alpha, po[q], omega, so[q]);
            r[k[q]] = rk;
            p_new[k[q]] = pk;
            const float vk = neu[q] ? pk : stencil_apply<2, float, false>(w[q], tile, lx[q], ly[q], 0);
            v_new[k[q]] = vk;
            dot[0].add(rh[q], vk);
            dot[1].add(rk, rk);
            dot[2].add(rh[q], rk);
        }
    }
    stage_drain(a, pp);
}

// Phase B from staged operands: s = r - alpha v (tile + halo), t = A s;
// dots t.s, t.t, s.s, r^.s, r^.t.
__device__ void phase_b2_staged(const PArgs &a, float *tile0, float *tile1, int parb, float alpha,
                                DotAcc<float> (&dot)[5], RowPipe<float> &pp) {
    using HD = HaloDims<2>;
    using TL = Tile<2>;
    const Geo &g = a.ta.g;
    float *s_out = (float *)a.s;
    float *t_out = (float *)a.t;
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    const int total = te - tb;
    if (tid == 0 && !pp.failed)
        for (int i = 0; i < Stage3::NB && i < total; ++i) stage_issue(a, pp, i, tb + i, false, parb);
    // alternate halo buffers, one __syncthreads per tile (as in phase CA)
    for (int i = 0; i < total; ++i) {
        const int b = i % Stage3::NB;
        float *tile = (i & 1) ? tile1 : tile0;
        stage_wait(a, pp, b);
        const unsigned char *st = reinterpret_cast<const unsigned char *>(pp.buf) + (size_t)b * Stage3::BYTES;
        const float *W = reinterpret_cast<const float *>(st);
        const float *R = reinterpret_cast<const float *>(st + Stage3::halo_off(0));
        const float *V = reinterpret_cast<const float *>(st + Stage3::halo_off(1));
        const float *RH = reinterpret_cast<const float *>(st + Stage3::point_off(0));
        int x0, y0, z0;
        tile_origin<2>(a.ta, tb + i, x0, y0, z0);
        int64_t k[TL::R];
        int lx[TL::R], ly[TL::R], lz[TL::R];
        bool neu[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            k[q] = tile_dp<2>(g, tid, q, x0, y0, z0, lx[q], ly[q], lz[q]);
            neu[q] = a.ta.kind && k[q] >= 0 && __ldg(a.ta.kind + k[q]) == KIND_NEUMANN;
        }
        for (int h = tid; h < HD::H; h += 256) {
            const int hy = h / HD::HX, hx = h - hy * HD::HX;
            const int hi = hy * Stage3::HXB + hx + 3;
            tile[h] = R[hi] - alpha * V[hi];
        }
        float w[TL::R][9], rh[TL::R];
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            const int pi = ly[q] * Stage3::TX + lx[q];
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) w[q][sl] = W[sl * (Stage3::TX * Stage3::TY) + pi];
            rh[q] = RH[pi];
        }
        __syncthreads();
        if (tid == 0 && !pp.failed && i + Stage3::NB < total) stage_issue(a, pp, b, tb + i + Stage3::NB, false, parb);
#pragma unroll
        for (int q = 0; q < TL::R; ++q) {
            if (k[q] < 0) continue;
            const float sk = tile[tile_centre<2>(lx[q], ly[q], 0)];
            s_out[k[q]] = sk;
            const float tk = neu[q] ? sk : stencil_apply<2, float, false>(w[q], tile, lx[q], ly[q], 0);
            t_out[k[q]] = tk;
            dot[0].add(tk, sk);
            dot[1].add(tk, tk);
            dot[2].add(sk, sk);
            dot[3].add(rh[q], sk);
            dot[4].add(rh[q], tk);
        }
    }
    stage_drain(a, pp);
}

// The scalar step of a true-residual update (block 0, thread 0), from the
// totals ||r64||^2, ||b||^2, r^.r, r.r (the last two in the recursion's
// precision) of r = b - A64 x64: convergence, and whether the recursion goes
// on with the replaced residual or restarts from it.
template <typename T>
__device__ void tr_last_update(Scalars *sc, const double *tot, double tol, int update_mode, int net_exit) {
    sc->rr64 = tot[0];
    sc->bb64 = tot[1];
    sc->rr = tot[3];
    sc->tol2 = tol * tol * tot[1];
    sc->pending = 0;
    if constexpr (sizeof(T) == 4) {
        sc->tol2_d = df_from(sc->tol2);
        sc->rr_d = df_from(tot[3]);
    }
    if (!isfinite(tot[0] + tot[1])) { sc->done = 4; return; }
    if (tot[0] <= sc->tol2) { sc->done = 1; return; }
    if (sc->max_hit) { sc->done = 2; return; }
    sc->rr_last = tot[3];
    sc->it_last = sc->iter;
    sc->updates += 1;
    // the recursion's scalars (kept as double-float pairs by the FP32
    // kernels)
    double rho_c = sc->rho, alpha_c = sc->alpha, omega_c = sc->omega;
    if constexpr (sizeof(T) == 4) {
        sc->rr_last_d = df_from(tot[3]);
        rho_c = df_value(sc->rho_d);
        alpha_c = df_value(sc->alpha_d);
        omega_c = df_value(sc->omega_d);
    }
    const bool corrected = sc->net_fresh != 0 || sc->discard != 0;
    const bool keep = update_mode == 2 && !sc->no_replace && !corrected && !sc->restart && !sc->s_conv &&
                      rho_c != 0.0 && omega_c != 0.0;
    // an update that restarts the recursion (the first, after a dropped
    // cycle, an ||s|| stop or a breakdown; every update of the restarting
    // schedule) begins a new refinement cycle: with a preconditioner network
    // the host adds the network's correction of this residual first
    // (done = 5) and relaunches with net_fresh set
    if (net_exit && !sc->net_fresh && !keep) { sc->done = 5; return; }
    sc->net_fresh = 0;
    sc->discard = 0;
    // residual replacement (update_mode 2): r now holds the true residual;
    // the recursion continues from the last complete iteration with beta
    // recomputed from rho' = r^.r, keeping p, v and r^.  Otherwise (update
    // mode 1, the first update, after an ||s|| stop or a restart) the
    // recursion restarts from r.
    if (keep) {
        const double beta = (tot[2] / rho_c) * (alpha_c / omega_c);
        if (isfinite(beta)) {
            sc->beta = beta;
            sc->replace = 1;
            if constexpr (sizeof(T) == 4)
                sc->beta_f = (float)beta;   // alpha_f, omega_f stay those of the last iteration
            else
                publish(sc);
            return;
        }
    }
    sc->restart = 1;
    sc->s_conv = 0;
    sc->alpha = sc->beta = sc->omega = 0.0;
    if constexpr (sizeof(T) == 4) sc->alpha_d = sc->omega_d = make_float2(0.0f, 0.0f);
    publish(sc);
}

// True-residual (reliable) update of the persistent two- and one-barrier
// kernels: fold the correction into x64 (or drop it after a diverged cycle),
// r_out = b - A64 x64 in the recursion's precision, then tr_last_update.
// False if a barrier wait gave up.
template <int G, typename T>
__device__ bool true_residual_update(const PArgs &a, unsigned &epoch, Scalars &ls, ScalarSnap<T> &snap, T *r_out) {
    if (a.mixed) {
        if (snap.discard)
            phase_discard<G, T>(a);
        else
            phase_fold<G, T>(a);
        DotAcc<double> none[1];
        if (!grid_reduce<1>(a, epoch, none, [&](double *) {})) return false;
    }
    DotAcc<double> d64[2];
    DotAcc<T> dt[2];
    phase_true_residual<G, T>(a, d64, dt, r_out);
    DotAcc<double> all[4];
    all[0].v = d64[0].v;
    all[1].v = d64[1].v;
    if constexpr (sizeof(T) == 4) {
        all[2].v = (double)dt[0].v.hi + (double)dt[0].v.lo;
        all[3].v = (double)dt[1].v.hi + (double)dt[1].v.lo;
    } else {
        all[2].v = dt[0].v;
        all[3].v = dt[1].v;
    }
    const double tol = a.tol;
    const int update_mode = a.update_mode;
    const int net_exit = a.net_exit;
    if (!grid_reduce<4>(a, epoch, all, [&](double *tot) {
            tr_last_update<T>(&ls, tot, tol, update_mode, net_exit);
            store_scalars(a.sc, ls);
        }))
        return false;
    take_scalars(a.sc, snap);
    return true;
}

// Wide stencils ask for two blocks per SM explicitly (their accumulators
// otherwise lead the register allocator to spill); a minimum of 0 leaves the
// compact stencils as the compiler places them.
template <int G, typename T>
__global__ void __launch_bounds__(256, Shape<G>::S > 27 ? 2 : 0) bicg_persistent2(const __grid_constant__ PArgs a) {
    using HD = HaloDims<G>;
    __shared__ T tile[HD::H];
    // the staged FP32 phases alternate between tile and tile_alt
    __shared__ T tile_alt[(G == 2 && sizeof(T) == 4) ? HD::H : 1];
    extern __shared__ __align__(128) unsigned char pipe_smem[];
    __shared__ __align__(8) uint64_t pipe_mbar[Shape<G>::S > 27 ? RowPipe<T>::NB : Stage3::NB];
    RowPipe<T> pp;
    pp.buf = reinterpret_cast<T *>(pipe_smem);
    pp.mbar = pipe_mbar;
    pp.parity = 0;
    pp.failed = false;
    pp.outstanding = 0;
    if constexpr (Shape<G>::S > 27) {
        if (a.tma_rows && threadIdx.x == 0) {
            for (int b = 0; b < RowPipe<T>::NB; ++b)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(pipe_mbar + b)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    } else if constexpr (G == 2 && sizeof(T) == 4) {
        if (a.tma3 && threadIdx.x == 0) {
            for (int b = 0; b < Stage3::NB; ++b)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(pipe_mbar + b)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    // Block 0 alone updates the scalars (in the barriers' `last` step), on a
    // copy in its shared memory (the tests and updates then read no global
    // memory), and writes the copy out before it releases the other blocks.
    __shared__ Scalars ls;
    if (threadIdx.x == 0) ls = *a.sc;
    Scalars *sc = &ls;
    int iters = 0;
    unsigned epoch = 0;
    // After each barrier thread 0 alone reads the scalars (it is the thread
    // that acquired the release) and hands them to its block through shared
    // memory.  When all 256 threads of every block read them, the
    // requests of about 2400 warps for the same two lines queue at one L2
    // slice, and the last blocks start their phase microseconds late.
    __shared__ ScalarSnap<T> snap;
    take_scalars(a.sc, snap);
    for (;;) {
        const int done0 = snap.done, perr0 = snap.perr, pend0 = snap.pend;
        const int par = snap.par, restart0 = snap.restart, sconv0 = snap.sconv, replace0 = snap.replace;
        const T alpha0 = snap.alpha, omega0 = snap.omega, beta0 = snap.beta;
        if (done0 || perr0) goto finish;
        if (pend0) {
            // ---- true residual (reliable) update
            if (!true_residual_update<G, T>(a, epoch, ls, snap, (T *)a.r)) goto finish;
            continue;
        }
        if (iters >= a.iter_budget) goto finish;
        const int it = iters;
        ++iters;
        stamp(a, it, 0);
        stamp_block_start(a, it);
        T *p_old = (T *)(par ? a.p1 : a.p0), *p_new = (T *)(par ? a.p0 : a.p1);
        T *v_old = (T *)(par ? a.v1 : a.v0), *v_new = (T *)(par ? a.v0 : a.v1);
        // ---- phase CA: x, r of the last iteration; p, v = A p; alpha ------
        {
            const int mode = restart0 ? CA_RESTART : (replace0 ? CA_REPLACE : (sconv0 ? CA_SCONV : CA_NORMAL));
            DotAcc<T> dot[3];
            if constexpr (G == 2 && sizeof(T) == 4) {
                if (a.tma3 && mode == CA_NORMAL)
                    phase_ca_staged(a, tile, tile_alt, par, alpha0, omega0, beta0, dot, pp);
                else
                    phase_ca<G, T>(a, tile, p_old, v_old, p_new, v_new, alpha0, omega0, beta0, mode, dot, pp);
            } else {
                phase_ca<G, T>(a, tile, p_old, v_old, p_new, v_new, alpha0, omega0, beta0, mode, dot, pp);
            }
            stamp(a, it, 1);
            stamp_block(a, it);
            const int stall = a.stall;
            const double eps = a.eps_breakdown;
            const double update2 = a.update2;
            const int mixed = a.mixed;
            const int update_mode_ca = a.update_mode;
            auto ca_last = [&](const double *tot) {
                const double rv = tot[0], rr = tot[1], rho = tot[2];
                sc->rv = rv;
                sc->rr = rr;
                sc->replace = 0;
                // iteration k finished (x, r); a replacement CA finishes none
                if (mode == CA_NORMAL || mode == CA_SCONV) sc->iter += 1;
                if (!isfinite(rv + rr + rho)) { sc->diverged = 5; sc->done = 4; return; }
                // s_conv stays set: the update that follows restarts (this
                // iteration computed no omega to continue from)
                if (mode == CA_SCONV) { sc->pending = 1; return; }
                if (mode == CA_RESTART) {
                    sc->rhat2 = rr;
                } else {
                    if (rr <= sc->tol2) { sc->pending = 1; return; }
                    if (sc->iter >= sc->max_iter) { sc->max_hit = 1; sc->pending = 1; return; }
                    if (mixed && rr <= update2 * sc->rr_last) { sc->pending = 1; return; }
                    // a recursion whose residual grew since the last true
                    // residual beyond what its schedule allows has diverged.
                    // Replacing residuals: the cycle's correction is dropped,
                    // the recursion restarts from the last folded iterate and
                    // every later update of the solve restarts.  Restarting:
                    // the solve finishes in FP64 from the last folded iterate.
                    // growth that counts as divergence: 100-fold in norm while
                    // residuals are replaced; the restarting schedule's short
                    // cycles spike higher on their own (1e4-fold)
                    const bool replacing = update_mode_ca == 2 && !sc->no_replace;
                    if (mixed && rr > (replacing ? 1e4 : 1e8) * sc->rr_last) {
                        sc->divergences += 1;
                        // the restarting schedule would rerun the same cycle
                        // bit for bit: its divergence ends the FP32 solve
                        if (!replacing) { sc->diverged = 1; sc->done = 3; return; }
                        sc->discard = 1;
                        sc->no_replace = 1;
                        sc->pending = 1;
                        return;
                    }
                    if (mixed && sc->iter - sc->it_last >= stall) { sc->pending = 1; return; }
                    // |rho| <= eps sqrt(|r^|^2 |r|^2), squared: no FP64
                    // square root on the barrier's path
                    if (rho * rho <= eps * eps * (sc->rhat2 * rr)) {
                        sc->restarts += 1;
                        if (sc->restarts > 1000) { sc->diverged = 2; sc->done = 3; return; }
                        sc->restart = 1;   // redo CA from this r with p = r
                        return;
                    }
                }
                sc->restart = 0;
                sc->parity ^= 1;
                sc->rho = rho;
                const double alpha_n = rho / rv;
                if (!isfinite(alpha_n) || alpha_n == 0.0) { sc->diverged = 3; sc->done = 3; return; }
                sc->alpha = alpha_n;
                sc->alpha_f = (float)alpha_n;   // omega_f and beta_f are unchanged since phase B
            };
            // the same tests and updates on the FP32 pipe (double-float
            // scalars; a threshold test reads the high word)
            auto ca_last_df = [&](const DF *tot) {
                const DF rv = df_norm(tot[0]), rr = df_norm(tot[1]), rho = df_norm(tot[2]);
                sc->rv_d = df_pack(rv);
                sc->rr_d = df_pack(rr);
                sc->replace = 0;
                if (mode == CA_NORMAL || mode == CA_SCONV) sc->iter += 1;
                if (!isfinite(rv.hi + rr.hi + rho.hi)) { sc->diverged = 5; sc->done = 4; return; }
                if (mode == CA_SCONV) { sc->pending = 1; return; }
                if (mode == CA_RESTART) {
                    sc->rhat2_d = df_pack(rr);
                } else {
                    const float rrf = rr.hi, last = sc->rr_last_d.x;
                    if (rrf <= sc->tol2_d.x) { sc->pending = 1; return; }
                    if (sc->iter >= sc->max_iter) { sc->max_hit = 1; sc->pending = 1; return; }
                    if (rrf <= (float)update2 * last) { sc->pending = 1; return; }
                    const bool replacing = update_mode_ca == 2 && !sc->no_replace;
                    if (rrf > (replacing ? 1e4f : 1e8f) * last) {
                        sc->divergences += 1;
                        if (!replacing) { sc->diverged = 1; sc->done = 3; return; }
                        sc->discard = 1;
                        sc->no_replace = 1;
                        sc->pending = 1;
                        return;
                    }
                    if (sc->iter - sc->it_last >= stall) { sc->pending = 1; return; }
                    if (fabsf(rho.hi) <= (float)eps * sqrtf(sc->rhat2_d.x) * sqrtf(rrf)) {
                        sc->restarts += 1;
                        if (sc->restarts > 1000) { sc->diverged = 2; sc->done = 3; return; }
                        sc->restart = 1;
                        return;
                    }
                }
                sc->restart = 0;
                sc->parity ^= 1;
                sc->rho_d = df_pack(rho);
                const DF alpha_n = df_div(rho, rv);
                if (!isfinite(alpha_n.hi) || alpha_n.hi == 0.0f) { sc->diverged = 3; sc->done = 3; return; }
                sc->alpha_d = df_pack(alpha_n);
                sc->alpha_f = alpha_n.hi;   // omega_f and beta_f are unchanged since phase B
            };
            bool ok;
            if constexpr (sizeof(T) == 4) {
                ok = grid_reduce_df<3>(a, epoch, dot, [&](const DF *tot) {
                    ca_last_df(tot);
                    store_step_scalars<T>(a.sc, ls);
                });
            } else {
                ok = grid_reduce<3>(a, epoch, dot, [&](double *tot) { ca_last(tot); store_step_scalars<T>(a.sc, ls); });
            }
            if (ok) take_scalars(a.sc, snap);
            if (!ok) goto finish;
            stamp(a, it, 2);
        }
        const int done1 = snap.done, pend1 = snap.pend, restart1 = snap.restart;
        const int parb = snap.par;
        const T alpha = snap.alpha;
        if (done1 || pend1 || restart1) continue;
        // ---- phase B: s, t = A s; omega, beta ------------------------------
        {
            const T *v_cur = (const T *)(parb ? a.v1 : a.v0);
            DotAcc<T> dot[5];
            if constexpr (G == 2 && sizeof(T) == 4) {
                if (a.tma3)
                    phase_b2_staged(a, tile, tile_alt, parb, alpha, dot, pp);
                else
                    phase_b2<G, T>(a, tile, v_cur, alpha, dot, pp);
            } else {
                phase_b2<G, T>(a, tile, v_cur, alpha, dot, pp);
            }
            stamp(a, it, 3);
            auto b_last = [&](const double *tot) {
                sc->ts = tot[0];
                sc->tt = tot[1];
                sc->ss = tot[2];
                if (!isfinite(tot[0] + tot[1] + tot[2] + tot[3] + tot[4])) { sc->diverged = 5; sc->done = 4; return; }
                if (tot[2] <= sc->tol2) { sc->s_conv = 1; return; }
                if (tot[1] == 0.0) { sc->diverged = 4; sc->done = 3; return; }
                const double omega = tot[0] / tot[1];
                const double rho_next = tot[3] - omega * tot[4];
                sc->omega = omega;
                sc->beta = (rho_next / sc->rho) * (sc->alpha / omega);
                publish(sc);
            };
            auto b_last_df = [&](const DF *tot_raw) {
                DF tot[5];
                for (int q = 0; q < 5; ++q) tot[q] = df_norm(tot_raw[q]);
                sc->ts_d = df_pack(tot[0]);
                sc->tt_d = df_pack(tot[1]);
                sc->ss_d = df_pack(tot[2]);
                if (!isfinite(tot[0].hi + tot[1].hi + tot[2].hi + tot[3].hi + tot[4].hi)) {
                    sc->diverged = 5;
                    sc->done = 4;
                    return;
                }
                if (tot[2].hi <= sc->tol2_d.x) { sc->s_conv = 1; return; }
                if (tot[1].hi == 0.0f) { sc->diverged = 4; sc->done = 3; return; }
                const DF omega = df_div(tot[0], tot[1]);
                const DF rho_next = df_sub(tot[3], df_mul(omega, tot[4]));
                const DF beta = df_mul(df_div(rho_next, df_unpack(sc->rho_d)), df_div(df_unpack(sc->alpha_d), omega));
                sc->omega_d = df_pack(omega);
                sc->omega_f = omega.hi;
                sc->beta_f = beta.hi;
            };
            bool ok;
            if constexpr (sizeof(T) == 4) {
                ok = grid_reduce_df<5>(a, epoch, dot, [&](const DF *tot) {
                    b_last_df(tot);
                    store_step_scalars<T>(a.sc, ls);
                });
            } else {
                ok = grid_reduce<5>(a, epoch, dot, [&](double *tot) { b_last(tot); store_step_scalars<T>(a.sc, ls); });
            }
            if (ok) take_scalars(a.sc, snap);
            if (!ok) goto finish;
            stamp(a, it, 4);
        }
    }
finish:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if constexpr (sizeof(T) == 4) {
            // the doubles the host reads for its diagnostics
            ls.rho = df_value(ls.rho_d);
            ls.alpha = df_value(ls.alpha_d);
            ls.omega = df_value(ls.omega_d);
            ls.rv = df_value(ls.rv_d);
            ls.rr = df_value(ls.rr_d);
            ls.rhat2 = df_value(ls.rhat2_d);
            ls.ts = df_value(ls.ts_d);
            ls.tt = df_value(ls.tt_d);
            ls.ss = df_value(ls.ss_d);
        }
        store_scalars(a.sc, ls);
    }
}

// ---- one grid barrier per iteration (2D 3x3 FP32, operands staged by TMA) --
// Bi-CGSTAB needs alpha before s = r - alpha v and t = A s, and omega
// before r' = s - omega t: two reductions per iteration in its textbook
// order.  Here each phase finishes iteration k and prepares iteration k+1
// up to its reduction, with three stencils instead of two:
//   x += alpha p + omega s,  r' = s - omega t     (s = r - alpha v, t = u - alpha q)
//   p' = r' + beta (p - omega v),  v' = A p',  q' = A v',  u' = A r'.
// t = A s = A r - alpha A v = u - alpha q holds for the stored u and q, so
// the dot products that fix omega and the next rho are polynomials in alpha
// of dot products of r', v', u', q', r^ from the same phase:
//   r^.v', r^.r', r'.r', u'.r', u'.v' + q'.r', q'.v', u'.u', u'.q', q'.q',
//   r^.u', r^.q'
// give alpha = r^.r' / r^.v' and, with s = r' - alpha v', t = u' - alpha q',
//   t.s = u'.r' - alpha (u'.v' + q'.r') + alpha^2 q'.v',
//   t.t = u'.u' - 2 alpha u'.q' + alpha^2 q'.q',
//   rho'' = r^.s - omega r^.t,
// so one reduction per iteration yields alpha, omega and beta.  alpha and
// the residual tests use direct dot products; omega and beta come from the
// polynomials, evaluated in double-float.  q' = A A p' carries the square of
// the rows' O(1 / l0^2) scale, and q'.q' would leave the FP32 range on fine
// meshes: q~ = sigma q' is stored instead, sigma = 2^k close to l0^2, and
// alpha~ = alpha / sigma multiplies it (both scalings exact), so
// t = u - alpha~ q~ and
//   t.t = u'.u' - 2 alpha~ u'.q~ + alpha~^2 q~.q~.  The phase needs p' two cells
// beyond the tile (v' one beyond, q' on it): each tile is staged with a
// two-cell halo of r, p, v, u, q and a one-cell halo of the rows.
struct Stage1 {
    static constexpr int TX = 32, TY = 16;
    static constexpr int WX = 40, WY = 18;    // rows box, from (x0 - 4, y0 - 1)
    static constexpr int HX = 40, HY = 20;    // vector boxes, from (x0 - 4, y0 - 2)
    static constexpr int WS = WX * WY;        // slot stride of the rows box
    static constexpr unsigned W_BYTES = 9u * WX * WY * 4u;   // 25920
    static constexpr unsigned W_PAD = 26112u;                 // 128-byte multiple
    static constexpr unsigned H_BYTES = HX * HY * 4u;         // 3200 (25 x 128)
    static constexpr unsigned P_BYTES = TX * TY * 4u;         // 2048
    static constexpr unsigned BYTES = W_PAD + 5u * H_BYTES + 3u * P_BYTES;
    static constexpr int NB = 2;
    static constexpr unsigned halo_off(int q) { return W_PAD + (unsigned)q * H_BYTES; }
    static constexpr unsigned point_off(int q) { return W_PAD + 5u * H_BYTES + (unsigned)q * P_BYTES; }
};
static_assert(Tile<2>::X == Stage1::TX && Tile<2>::Y == Stage1::TY, "stage boxes are one 2D tile");
static_assert(Stage1::BYTES % 128 == 0 && Stage1::W_PAD >= Stage1::W_BYTES, "128-byte aligned stage buffers");
enum { B1_R = 0, B1_P = 1, B1_V = 2, B1_U = 3, B1_Q = 4 };
enum { ONE_NORMAL = 0, ONE_REPLACE = 1, ONE_RESTART = 2 };

// Copies of one tile for a phase of mode `mode` reading buffer pair `par`:
// normal r, p, v, u, q halos and r^, x, xlo; replacement (r holds the true
// residual) r, p, v and r^; restart r alone.
__device__ __forceinline__ unsigned stage1_tx(int mode) {
    return Stage1::W_BYTES + (mode == ONE_NORMAL ? 5u * Stage1::H_BYTES + 3u * Stage1::P_BYTES
                              : mode == ONE_REPLACE ? 3u * Stage1::H_BYTES + Stage1::P_BYTES
                                                    : Stage1::H_BYTES);
}

__device__ __forceinline__ void stage1_issue(const PArgs &a, RowPipe<float> &pp, int b, int tl, int mode, int par) {
    pp.outstanding |= 1u << b;
    int x0, y0, z0;
    tile_origin<2>(a.ta, tl, x0, y0, z0);
    const uint32_t mb = smem_addr(pp.mbar + b);
    const uint32_t dst = smem_addr(pp.buf) + (uint32_t)b * Stage1::BYTES;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads and writes of the buffer
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(stage1_tx(mode)) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(&a.maps1.rows)), "r"(x0 - 4), "r"(y0 - 1), "r"(0), "r"(mb)
        : "memory");
    const int hx = x0 - 4, hy = y0 - 2;
    tma_2d(dst + Stage1::halo_off(B1_R), &a.maps1.vec[0 + par], hx, hy, mb);
    if (mode == ONE_RESTART) return;
    tma_2d(dst + Stage1::halo_off(B1_P), &a.maps1.vec[2 + par], hx, hy, mb);
    tma_2d(dst + Stage1::halo_off(B1_V), &a.maps1.vec[4 + par], hx, hy, mb);
    tma_2d(dst + Stage1::point_off(PT_RH), &a.maps3.point[PT_RH], x0, y0, mb);
    if (mode == ONE_REPLACE) return;
    tma_2d(dst + Stage1::halo_off(B1_U), &a.maps1.vec[6 + par], hx, hy, mb);
    tma_2d(dst + Stage1::halo_off(B1_Q), &a.maps1.vec[8 + par], hx, hy, mb);
    tma_2d(dst + Stage1::point_off(PT_X), &a.maps3.point[PT_X], x0, y0, mb);
    tma_2d(dst + Stage1::point_off(PT_XLO), &a.maps3.point[PT_XLO], x0, y0, mb);
}

// (A y)_k of the FP32 difference-form row whose weights sit in the staged
// rows box at wi and y in a vector box (row stride 40) at yi: the
// compensated sum of stencil_apply, term for term in the same order.
__device__ __forceinline__ float box_stencil(const float *W, int wi, const float *Y, int yi) {
    const float yk = Y[yi];
    float hi = W[4 * Stage1::WS + wi] * yk, lo = 0.0f;   // centre weight is 0 or 1: exact
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        if (s == 4) continue;
        const int o = (s % 3 - 1) + Stage1::HX * (s / 3 - 1);
        const float w = W[s * Stage1::WS + wi];
        const float d = __fsub_rn(Y[yi + o], yk);
        const float p = __fmul_rn(w, d);
        const float pe = __fmaf_rn(w, d, -p);
        float e;
        two_sum(hi, p, hi, e);
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    return __fadd_rn(hi, lo);
}

// One phase of the one-barrier schedule over the block's tiles.  Reads the
// buffers of parity par, writes those of par ^ 1 (r', p', v', u', q'; r^ on
// a restart) and the correction x, xlo.  Dot products as listed above.
__device__ void phase_one(const PArgs &a, int par, int mode, float alpha, float omega, float beta,
                          DotAcc<float> (&dot)[11], RowPipe<float> &pp) {
    const Geo &g = a.ta.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const int np = par ^ 1;
    float *x = (float *)a.x;
    float *r_new = (float *)(np ? a.r1 : a.r);
    float *p_new = (float *)(np ? a.p1 : a.p0);
    float *v_new = (float *)(np ? a.v1 : a.v0);
    float *u_new = (float *)(np ? a.u1 : a.u0);
    float *q_new = (float *)(np ? a.q1 : a.q0);
    float *rh_out = (float *)a.rh;
    const int8_t *kind = a.ta.kind;
    const float qs = a.q_scale, qu = a.q_unscale;
    const float alpha_q = alpha * qu;   // exact: qu is a power of two
    const int tid = threadIdx.x;
    const int tb = tile_first(a, blockIdx.x), te = tile_first(a, blockIdx.x + 1);
    const int total = te - tb;
    if (tid == 0 && !pp.failed)
        for (int i = 0; i < Stage1::NB && i < total; ++i) stage1_issue(a, pp, i, tb + i, mode, par);
    for (int i = 0; i < total; ++i) {
        const int b = i % Stage1::NB;
        stage_wait(a, pp, b);
        unsigned char *st = reinterpret_cast<unsigned char *>(pp.buf) + (size_t)b * Stage1::BYTES;
        const float *W = reinterpret_cast<const float *>(st);
        float *R = reinterpret_cast<float *>(st + Stage1::halo_off(B1_R));
        float *P = reinterpret_cast<float *>(st + Stage1::halo_off(B1_P));
        float *V = reinterpret_cast<float *>(st + Stage1::halo_off(B1_V));
        const float *U = reinterpret_cast<const float *>(st + Stage1::halo_off(B1_U));
        const float *Q = reinterpret_cast<const float *>(st + Stage1::halo_off(B1_Q));
        const float *RH = reinterpret_cast<const float *>(st + Stage1::point_off(PT_RH));
        const float *X = reinterpret_cast<const float *>(st + Stage1::point_off(PT_X));
        const float *XL = reinterpret_cast<const float *>(st + Stage1::point_off(PT_XLO));
        int x0, y0, z0;
        tile_origin<2>(a.ta, tb + i, x0, y0, z0);
        // (1) r' and p' on the tile and two rings of halo (in place); the
        // tile's correction, r' and p'.  Cells past the mesh hold zeros.
        for (int h = tid; h < 36 * 20; h += 256) {
            const int hy = h / 36, hx = h - hy * 36;
            const int bi = hy * Stage1::HX + hx + 2;
            const float rk = R[bi];
            float rn = rk, pn = rk, sk = 0.0f, pk = 0.0f;
            if (mode != ONE_RESTART) {
                const float vk = V[bi];
                pk = P[bi];
                if (mode == ONE_NORMAL) {
                    sk = __fmaf_rn(-alpha, vk, rk);
                    const float tk = __fmaf_rn(-alpha_q, Q[bi], U[bi]);
                    rn = __fmaf_rn(-omega, tk, sk);
                }
                pn = __fmaf_rn(beta, __fmaf_rn(-omega, vk, pk), rn);
            }
            const int lx = hx - 2, ly = hy - 2;
            if (lx >= 0 && lx < Stage1::TX && ly >= 0 && ly < Stage1::TY && x0 + lx < n0 && y0 + ly < n1) {
                const int64_t k = (int64_t)(x0 + lx) + (int64_t)n0 * (y0 + ly);
                const int pi = ly * Stage1::TX + lx;
                if (mode == ONE_NORMAL) add_correction(a.xlo, x, k, X[pi], XL[pi], alpha, pk, omega, sk);
                r_new[k] = rn;
                p_new[k] = pn;
                if (mode == ONE_RESTART) rh_out[k] = rn;
            }
            R[bi] = rn;
            P[bi] = pn;
        }
        __syncthreads();
        // (2) v' = A p' on the tile and one ring of halo (into the v box)
        for (int h = tid; h < 34 * 18; h += 256) {
            const int hy = h / 34, hx = h - hy * 34;
            const int bi = (hy + 1) * Stage1::HX + hx + 3;
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
            float vn = 0.0f;
            if (gx >= 0 && gx < n0 && gy >= 0 && gy < n1) {
                const int64_t k = (int64_t)gx + (int64_t)n0 * gy;
                vn = (kind && kind[k] == KIND_NEUMANN) ? P[bi] : box_stencil(W, hy * Stage1::WX + hx + 3, P, bi);
            }
            V[bi] = vn;
        }
        __syncthreads();
        // (3) the tile: q' = A v', u' = A r', stores and dot products
#pragma unroll
        for (int c0 = 0; c0 < Stage1::TX * Stage1::TY; c0 += 256) {
            const int c = c0 + tid;
            const int lx = c % Stage1::TX, ly = c / Stage1::TX;
            if (x0 + lx >= n0 || y0 + ly >= n1) continue;
            const int64_t k = (int64_t)(x0 + lx) + (int64_t)n0 * (y0 + ly);
            const int bi = (ly + 2) * Stage1::HX + lx + 4;
            const int wi = (ly + 1) * Stage1::WX + lx + 4;
            const float vk = V[bi], rk = R[bi];
            const bool neu = kind && kind[k] == KIND_NEUMANN;
            const float qk = qs * (neu ? vk : box_stencil(W, wi, V, bi));   // q~ = sigma A v'
            const float uk = (mode == ONE_RESTART || neu) ? (mode == ONE_RESTART ? vk : rk) : box_stencil(W, wi, R, bi);
            v_new[k] = vk;
            q_new[k] = qk;
            u_new[k] = uk;
            const float rh = (mode == ONE_RESTART) ? rk : RH[ly * Stage1::TX + lx];
            dot[0].add(rh, vk);
            dot[1].add(rh, rk);
            dot[2].add(rk, rk);
            dot[3].add(uk, rk);
            dot[4].add(uk, vk);
            dot[4].add(qk * qu, rk);   // q'.r' itself: its size is that of u'.v'
            dot[5].add(qk, vk);
            dot[6].add(uk, uk);
            dot[7].add(uk, qk);
            dot[8].add(qk, qk);
            dot[9].add(rh, uk);
            dot[10].add(rh, qk);
        }
        __syncthreads();   // stage b is read: refill it
        if (tid == 0 && !pp.failed && i + Stage1::NB < total) stage1_issue(a, pp, b, tb + i + Stage1::NB, mode, par);
    }
    stage_drain(a, pp);
}

__global__ void __launch_bounds__(256, 2) bicg_persistent1(const __grid_constant__ PArgs a) {
    extern __shared__ __align__(128) unsigned char pipe_smem[];
    __shared__ __align__(8) uint64_t pipe_mbar[Stage1::NB];
    RowPipe<float> pp;
    pp.buf = reinterpret_cast<float *>(pipe_smem);
    pp.mbar = pipe_mbar;
    pp.parity = 0;
    pp.failed = false;
    pp.outstanding = 0;
    if (threadIdx.x == 0) {
        for (int b = 0; b < Stage1::NB; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(pipe_mbar + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // block 0 updates its shared-memory copy of the scalars, as in
    // bicg_persistent2
    __shared__ Scalars ls;
    if (threadIdx.x == 0) ls = *a.sc;
    Scalars *sc = &ls;
    int iters = 0;
    unsigned epoch = 0;
    __shared__ ScalarSnap<float> snap;
    take_scalars(a.sc, snap);
    for (;;) {
        if (snap.done || snap.perr) goto finish;
        const int par = snap.par;
        if (snap.pend) {
            // true residual into the r buffer the next phase reads
            if (!true_residual_update<2, float>(a, epoch, ls, snap, (float *)(par ? a.r1 : a.r))) goto finish;
            continue;
        }
        if (iters >= a.iter_budget) goto finish;
        const int it = iters;
        ++iters;
        stamp(a, it, 0);
        stamp_block_start(a, it);
        const int mode = snap.restart ? ONE_RESTART : (snap.replace ? ONE_REPLACE : ONE_NORMAL);
        DotAcc<float> dot[11];
        phase_one(a, par, mode, snap.alpha, snap.omega, snap.beta, dot, pp);
        stamp(a, it, 1);
        stamp_block(a, it);
        const int stall = a.stall;
        const float eps = (float)a.eps_breakdown;
        const float update2 = (float)a.update2;
        const int update_mode = a.update_mode;
        const float q_unscale = a.q_unscale;
        auto one_last = [&](const DF *raw) {
            DF t[11];
#pragma unroll
            for (int q = 0; q < 11; ++q) t[q] = df_norm(raw[q]);
            const DF rv = t[0], rho = t[1], rr = t[2];
            sc->rv_d = df_pack(rv);
            sc->rr_d = df_pack(rr);
            sc->replace = 0;
            // a normal phase completes an iteration (x and r'); a replaced
            // or restarted one only rebuilds the directions
            if (mode == ONE_NORMAL) sc->iter += 1;
            bool fin = true;
#pragma unroll
            for (int q = 0; q < 11; ++q) fin = fin && isfinite(t[q].hi);
            if (!fin) { sc->diverged = 5; sc->done = 4; return; }
            if (mode == ONE_RESTART) {
                sc->rhat2_d = df_pack(rr);
            } else {
                // the tests of bicg_persistent2 on r' (x is up to date: a
                // true-residual update may follow at once)
                const float rrf = rr.hi, last = sc->rr_last_d.x;
                if (rrf <= sc->tol2_d.x) { sc->pending = 1; return; }
                if (sc->iter >= sc->max_iter) { sc->max_hit = 1; sc->pending = 1; return; }
                if (rrf <= update2 * last) { sc->pending = 1; return; }
                const bool replacing = update_mode == 2 && !sc->no_replace;
                if (rrf > (replacing ? 1e4f : 1e8f) * last) {
                    sc->divergences += 1;
                    if (!replacing) { sc->diverged = 1; sc->done = 3; return; }
                    sc->discard = 1;
                    sc->no_replace = 1;
                    sc->pending = 1;
                    return;
                }
                if (sc->iter - sc->it_last >= stall) { sc->pending = 1; return; }
                if (fabsf(rho.hi) <= eps * sqrtf(sc->rhat2_d.x) * sqrtf(rrf)) {
                    sc->restarts += 1;
                    if (sc->restarts > 1000) { sc->diverged = 2; sc->done = 3; return; }
                    sc->restart = 1;
                    sc->parity ^= 1;   // restart from the r' this phase wrote
                    return;
                }
            }
            sc->restart = 0;
            sc->parity ^= 1;
            const DF alpha = df_div(rho, rv);
            if (!isfinite(alpha.hi) || alpha.hi == 0.0f) { sc->diverged = 3; sc->done = 3; return; }
            // alpha~ = alpha / sigma: t[5], t[7], t[8], t[10] hold dot
            // products with q~ = sigma q'
            const DF alq = DF{alpha.hi * q_unscale, alpha.lo * q_unscale};
            const DF ts = df_norm(df_add(df_sub(t[3], df_mul(alpha, t[4])), df_mul(alpha, df_mul(alq, t[5]))));
            const DF tt = df_norm(df_add(df_sub(t[6], df_mul(DF{2.0f * alq.hi, 2.0f * alq.lo}, t[7])),
                                         df_mul(df_mul(alq, alq), t[8])));
            sc->rho_d = df_pack(rho);
            sc->alpha_d = df_pack(alpha);
            sc->alpha_f = alpha.hi;
            sc->ts_d = df_pack(ts);
            sc->tt_d = df_pack(tt);
            if (!(tt.hi > 0.0f)) {
                // t = A s vanishes to rounding, so s does: the next phase
                // takes r'' = s and the residual tests follow
                sc->omega_d = make_float2(0.0f, 0.0f);
                sc->omega_f = 0.0f;
                sc->beta_f = 0.0f;
                return;
            }
            const DF omega = df_div(ts, tt);
            const DF rs = df_sub(rho, df_mul(alpha, rv));        // r^.s
            const DF rt = df_sub(t[9], df_mul(alq, t[10]));      // r^.t
            const DF rho_next = df_sub(rs, df_mul(omega, rt));
            const DF beta = df_mul(df_div(rho_next, rho), df_div(alpha, omega));
            sc->omega_d = df_pack(omega);
            sc->omega_f = omega.hi;
            sc->beta_f = beta.hi;
        };
        if (!grid_reduce_df<11>(a, epoch, dot, [&](const DF *tot) {
                one_last(tot);
                store_step_scalars<float>(a.sc, ls);
            }))
            goto finish;
        take_scalars(a.sc, snap);
        stamp(a, it, 2);
    }
finish:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ls.rho = df_value(ls.rho_d);
        ls.alpha = df_value(ls.alpha_d);
        ls.omega = df_value(ls.omega_d);
        ls.rv = df_value(ls.rv_d);
        ls.rr = df_value(ls.rr_d);
        ls.rhat2 = df_value(ls.rhat2_d);
        ls.ts = df_value(ls.ts_d);
        ls.tt = df_value(ls.tt_d);
        ls.ss = df_value(ls.ss_d);
        store_scalars(a.sc, ls);
    }
}

// Grid of the persistent launch: every resident slot (at most one block per
// tile).
// Dynamic shared memory of the two-barrier kernel: the TMA row buffers of a
// wide stencil, none otherwise.
template <int G, typename T>
static size_t pipe_smem_bytes(bool tma) {
    if (!tma) return 0;
    if (Shape<G>::S > 27) return (size_t)RowPipe<T>::NB * RowPipe<T>::BYTES;
    if (G == 2 && sizeof(T) == 4) return (size_t)Stage3::NB * Stage3::BYTES;
    return 0;
}

template <int G, typename T, int B>
static int persistent_grid(int ntiles, bool tma) {
    static const int occ3 = occupancy(bicg_persistent<G, T>);
    static int occ2[2] = {0, 0};
    int occ = occ3;
    if (B == 2) {
        int &o = occ2[tma ? 1 : 0];
        if (!o) {
            const size_t dyn = pipe_smem_bytes<G, T>(tma);
            if (dyn) cudaFuncSetAttribute(bicg_persistent2<G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            int blocks = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, bicg_persistent2<G, T>, 256, dyn) != cudaSuccess ||
                blocks < 1)
                blocks = 1;
            o = blocks;
        }
        occ = o;
    }
    const int maxg = std::max(1, occ * sm_count());
    return std::min(ntiles, maxg);
}

// Tensor map of the rows as a [S][n_y][n_x] tensor with a box of one tile
// by 9 slots, for the TMA row stream of wide stencils.  False when
// TMA cannot be used: a row stride or the slot stride is not a multiple of
// 16 bytes, or the driver does not provide the encoder.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int G, typename T>
static bool encode_row_map(const Geo &g, const void *row, CUtensorMap *map) {
    if (Shape<G>::S <= 27) return false;
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    if (!fn) return false;
    const uint64_t esz = sizeof(T);
    const uint64_t nx = (uint64_t)g.n[0], ny = (uint64_t)g.n[1];
    if ((nx * esz) % 16 != 0 || (nx * ny * esz) % 16 != 0 || ((uintptr_t)row % 16) != 0) return false;
    const cuuint64_t dims[3] = {nx, ny, (cuuint64_t)Shape<G>::S};
    const cuuint64_t strides[2] = {nx * esz, nx * ny * esz};
    const cuuint32_t box[3] = {(cuuint32_t)Tile<G>::X, (cuuint32_t)Tile<G>::Y, (cuuint32_t)RowPipe<T>::SL};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                          const_cast<void *>(row), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Process-wide switch of the staged phases (mcd_solver_set_staging).
static int g_no_stage = 0;
static bool st_no_stage() { return g_no_stage != 0; }

// Tensor maps of the staged 2D 3x3 FP32 phases: the rows as [9][n_y][n_x]
// (box 32 x 16 x 9), the halo vectors with a 40 x 18 box, the point vectors
// with a 32 x 16 box.  False (the phases then load directly) on a periodic
// mesh (a copy cannot wrap), when n_x is not a multiple of 4 (16-byte row
// strides), on meshes smaller than a halo box, or without the encoder.
static bool encode_stage_maps(const Geo &g, const float *row, const void *const *halo, const void *const *point,
                              PArgs &a) {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    if (!fn || g.dim != 2 || g.per[0] || g.per[1] || g.n[0] % 4 != 0) return false;
    if (g.n[0] < Stage3::HXB || g.n[1] < Stage3::HYB) return false;
    const cuuint64_t nx = (cuuint64_t)g.n[0], ny = (cuuint64_t)g.n[1];
    const cuuint32_t ones[3] = {1, 1, 1};
    auto aligned = [](const void *p) { return ((uintptr_t)p % 16) == 0; };
    {
        if (!aligned(row)) return false;
        const cuuint64_t dims[3] = {nx, ny, 9};
        const cuuint64_t str[2] = {nx * 4, nx * ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)Stage3::TX, (cuuint32_t)Stage3::TY, 9};
        if (fn(&a.maps3.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(row), dims, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    const cuuint64_t dims[2] = {nx, ny};
    const cuuint64_t str[1] = {nx * 4};
    for (int q = 0; q < 7 + 3; ++q) {
        const void *ptr = q < 7 ? halo[q] : point[q - 7];
        if (!ptr || !aligned(ptr)) return false;
        const cuuint32_t hbox[2] = {(cuuint32_t)Stage3::HXB, (cuuint32_t)Stage3::HYB};
        const cuuint32_t pbox[2] = {(cuuint32_t)Stage3::TX, (cuuint32_t)Stage3::TY};
        CUtensorMap *m = q < 7 ? &a.maps3.halo[q] : &a.maps3.point[q - 7];
        if (fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, str, q < 7 ? hbox : pbox, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// Tensor maps of the one-barrier kernel: the rows as [9][n_y][n_x] with a
// 40 x 18 x 9 box (the tile and one ring of halo, from x0 - 4 so that the
// copy starts on a 16-byte boundary) and the ten vectors with a 40 x 20 box
// (two rings).  Needs what encode_stage_maps needs and a mesh of at least
// 40 x 20 cells.
static bool encode_one_maps(const Geo &g, const float *row, const void *const *vec, PArgs &a) {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    if (!fn || g.dim != 2 || g.per[0] || g.per[1] || g.n[0] % 4 != 0) return false;
    if (g.n[0] < Stage1::HX || g.n[1] < Stage1::HY) return false;
    const cuuint64_t nx = (cuuint64_t)g.n[0], ny = (cuuint64_t)g.n[1];
    const cuuint32_t ones[3] = {1, 1, 1};
    auto aligned = [](const void *p) { return p && ((uintptr_t)p % 16) == 0; };
    if (!aligned(row)) return false;
    {
        const cuuint64_t dims[3] = {nx, ny, 9};
        const cuuint64_t str[2] = {nx * 4, nx * ny * 4};
        const cuuint32_t box[3] = {(cuuint32_t)Stage1::WX, (cuuint32_t)Stage1::WY, 9};
        if (fn(&a.maps1.rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(row), dims, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    const cuuint64_t dims[2] = {nx, ny};
    const cuuint64_t str[1] = {nx * 4};
    const cuuint32_t box[2] = {(cuuint32_t)Stage1::HX, (cuuint32_t)Stage1::HY};
    for (int q = 0; q < 10; ++q) {
        if (!aligned(vec[q])) return false;
        if (fn(&a.maps1.vec[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(vec[q]), dims, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// Grid of the one-barrier kernel: every resident slot (at most one block
// per tile).
static int persistent_grid_one(int ntiles) {
    static int occ = 0;
    if (!occ) {
        const size_t dyn = (size_t)Stage1::NB * Stage1::BYTES;
        cudaFuncSetAttribute(bicg_persistent1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, bicg_persistent1, 256, dyn) != cudaSuccess ||
            blocks < 1)
            blocks = 1;
        occ = blocks;
    }
    return std::min(ntiles, std::max(1, occ * sm_count()));
}

// Run the whole solve in persistent launches (each bounded by an iteration
// budget and the barrier spin limit).  On return w->h_sc holds the final
// scalars.  x64 is the FP64 solution; in FP64 mode it is also the iterate.
// Phase trace buffer (instrumentation; NULL unless mcd_trace_enable(1)).
static unsigned long long *g_trace = nullptr;

template <int G, typename T>
static mcd_status run_persistent(const mcd_stencils *st, double *x64, const mcd_solve_params *prm,
                                 mcd_status &result, int &net_corrections, cudaStream_t stream) {
    Workspace *w = st->ws;
    const Geo &g = st->geo;
    const bool mixed = sizeof(T) == 4;
    PArgs a;
    a.ta.g = g;
    a.ta.bx = (g.n[0] + Tile<G>::X - 1) / Tile<G>::X;
    a.ta.by = (g.n[1] + Tile<G>::Y - 1) / Tile<G>::Y;
    a.ta.bz = (Shape<G>::dim == 3) ? (g.n[2] + Tile<G>::Z - 1) / Tile<G>::Z : 1;
    a.ta.ntiles = a.ta.bx * a.ta.by * a.ta.bz;
    a.ta.kind = st->has_neumann ? st->kind : nullptr;
    const bool two = prm->barriers != 3;   // default: the two-barrier schedule
    memset(&a.tmap_rows, 0, sizeof(a.tmap_rows));
    a.tma_rows = (two && encode_row_map<G, T>(g, mixed ? (const void *)st->row32 : (const void *)st->row64,
                                               &a.tmap_rows))
                     ? 1
                     : 0;
    a.tma3 = 0;
    if (G == 2 && mixed && two && !st_no_stage()) {
        const void *halo[7] = {w->fs, w->ft, w->fp[0], w->fp[1], w->fv[0], w->fv[1], w->fr};
        const void *point[3] = {w->frh, w->fd, w->fdlo};
        a.tma3 = encode_stage_maps(g, st->row32, halo, point, a) ? 1 : 0;
    }
    const bool staged = a.tma_rows != 0 || a.tma3 != 0;
    // one grid barrier per iteration on request (barriers = 1) where the
    // staged 2D 3x3 FP32 phases run.  Not the default: its phase does more
    // work per tile than the two phases it replaces (three stencils and a
    // deeper halo), and on the 1024^2 cylinder an iteration took 56.6 us
    // against 52.0 us for the two-barrier schedule on the same GPU
    a.one = 0;
    if (G == 2 && mixed && a.tma3 && prm->barriers == 1 && w->fr1) {
        const void *vec[10] = {w->fr, w->fr1, w->fp[0], w->fp[1], w->fv[0], w->fv[1], w->fs, w->fu1, w->ft, w->fq1};
        a.one = encode_one_maps(g, st->row32, vec, a) ? 1 : 0;
    }
    a.q_scale = ldexpf(1.0f, (int)std::lround(std::log2(g.l0 * g.l0)));
    a.q_unscale = 1.0f / a.q_scale;
    a.r1 = w->fr1;
    a.u0 = w->fs;
    a.u1 = w->fu1;
    a.q0 = w->ft;
    a.q1 = w->fq1;
    const size_t dyn_smem = a.one ? (size_t)Stage1::NB * Stage1::BYTES : two ? pipe_smem_bytes<G, T>(staged) : 0;
    const int grid = a.one ? persistent_grid_one(a.ta.ntiles)
                     : two ? persistent_grid<G, T, 2>(a.ta.ntiles, staged)
                           : persistent_grid<G, T, 3>(a.ta.ntiles, false);
    a.grid = grid;
    a.row64 = st->row64;
    a.b = w->b;
    a.x64 = x64;
    if (mixed) {
        a.row = st->row32;
        a.x = w->fd; a.r = w->fr; a.rh = w->frh;
        a.xlo = two ? w->fdlo : nullptr;
        a.p0 = w->fp[0]; a.p1 = w->fp[1]; a.v0 = w->fv[0]; a.v1 = w->fv[1];
        a.s = w->fs; a.t = w->ft;
        MCD_CUDA_TRY(cudaMemsetAsync(w->fd, 0, g.N * sizeof(float), stream));
        MCD_CUDA_TRY(cudaMemsetAsync(w->fdlo, 0, g.N * sizeof(float), stream));
    } else {
        a.xlo = nullptr;
        a.row = st->row64;
        a.x = x64; a.r = w->dr; a.rh = w->drh;
        a.p0 = w->dp[0]; a.p1 = w->dp[1]; a.v0 = w->dv[0]; a.v1 = w->dv[1];
        a.s = w->ds; a.t = w->dt;
    }
    a.sc = w->sc;
    a.partials = w->partials;
    a.pstride = w->pstride;
    a.bar = w->bar;
    a.mixed = mixed ? 1 : 0;
    a.update_mode = mixed ? (prm->update_restart == 1 ? 1 : 2) : 1;
    const double upd = (prm->inner_tol > 0.0 && prm->inner_tol < 1.0) ? prm->inner_tol : 0.3;
    a.update2 = upd * upd;
    a.stall = 1024;
    a.tol = prm->tol;
    a.eps_breakdown = mixed ? 1e-12 : 1e-14;
    a.iter_budget = 4096;
    a.spin_limit = 1ll << 21;   // about 1.5 s of polls (L2 round trip + 64 ns sleep)
    a.trace = g_trace;
    a.net_exit = (mixed && two && prm->precond) ? 1 : 0;
    const size_t bar_bytes = barrier_bytes(grid);
    // start with a true-residual update of the initial guess
    int one = 1;
    MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->pending, &one, sizeof(int), cudaMemcpyHostToDevice, stream));
    MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->restart, &one, sizeof(int), cudaMemcpyHostToDevice, stream));
    const int max_launch = std::max(2, prm->max_iter / a.iter_budget + 8);
    for (int launch = 0;; ++launch) {
        void *args[] = {&a};
        MCD_CUDA_TRY(cudaMemsetAsync(w->bar, 0, bar_bytes, stream));
        {
            KTimer kt(MCD_K_SOLVE, stream);
            const void *kern = a.one ? (const void *)bicg_persistent1
                               : two ? (const void *)bicg_persistent2<G, T>
                                     : (const void *)bicg_persistent<G, T>;
            MCD_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(256), args, dyn_smem, stream));
        }
        mcd_status s = read_scalars(w, stream);
        if (s != MCD_OK) return s;
        const Scalars &h = *w->h_sc;
        if (h.phase_err) { result = MCD_ETIMEOUT; return MCD_OK; }
        if (h.done == 5) {
            // d0 of this refinement: the network's correction of the FP64
            // residual b - A x64, along its residual-minimising step.  A
            // correction that cuts the residual by less than 10 % ends the
            // network's part in this solve (the plain solve goes on)
            double ns[8] = {0.0};
            s = net_warm_start(prm->precond, st, w->b, nullptr, x64, ns, stream);
            if (s != MCD_OK) return s;
            net_corrections += 1;
            if (!(ns[4] > 0.0 && ns[6] < 0.81 * ns[3])) a.net_exit = 0;
            const int zero = 0;
            MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->done, &zero, sizeof(int), cudaMemcpyHostToDevice, stream));
            MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->pending, &one, sizeof(int), cudaMemcpyHostToDevice, stream));
            MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->restart, &one, sizeof(int), cudaMemcpyHostToDevice, stream));
            MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->net_fresh, &one, sizeof(int), cudaMemcpyHostToDevice, stream));
            --launch;   // not a launch of the iteration budget: every cycle runs >= 1 iteration
            continue;
        }
        if (h.done == 1) { result = MCD_OK; return MCD_OK; }
        if (h.done == 2) { result = MCD_ENOCONV; return MCD_OK; }
        if (h.done == 3) { result = MCD_EBREAKDOWN; return MCD_OK; }
        if (h.done == 4) { result = MCD_ENONFINITE; return MCD_OK; }
        if (launch >= max_launch) {
            set_error("persistent solve exceeded its launch budget");
            result = MCD_ENOCONV;
            return MCD_OK;
        }
    }
}

template <int G>
static mcd_status solve_impl(const mcd_stencils *st, const double *rhs, const double *bnd, double *p,
                             const mcd_solve_params *prm, mcd_solve_info *info, cudaStream_t stream) {
    Workspace *w = st->ws;
    const int64_t N = st->geo.N;
    mcd_status s = mcd_assemble_rhs(st, rhs, bnd, w->b, stream);
    if (s != MCD_OK) return s;
    if (prm->net && prm->net_dprev) {
        s = net_save_guess(prm->net, st, p, stream);
        if (s != MCD_OK) return s;
    }
    Scalars init;
    memset(&init, 0, sizeof(init));
    init.max_iter = prm->max_iter > 0 ? prm->max_iter : 1 << 30;
    MCD_CUDA_TRY(cudaMemcpyAsync(w->sc, &init, sizeof(init), cudaMemcpyHostToDevice, stream));
    MCD_KLAUNCH(MCD_K_OTHER, stream, fix_guess<<<w->nblk1, 256, 0, stream>>>(N, st->kind, w->b, p, w->sc));
    MCD_LAUNCH_CHECK();
    double ws_sc[8] = {0.0};
    if (prm->net) {
        s = net_warm_start(prm->net, st, w->b, prm->net_dprev, p, ws_sc, stream);
        if (s != MCD_OK) return s;
    }
    const int check_every = prm->check_every > 0 ? prm->check_every : 64;   // legacy schedule
    const int max_outer = prm->max_refine > 0 ? prm->max_refine : 50;
    const int max_launch = (init.max_iter > (1 << 29) ? (1 << 29) : init.max_iter) + 2 * check_every;

    mcd_status result = MCD_ENOCONV;
    int outer = 0;
    int mixed_iters = 0, fallback = 0, net_corr = 0, mixed_div = 0, mixed_upd = 0;
    if (prm->check_every >= 0) {
        // persistent cooperative solve (the default)
        s = (prm->mode == MCD_FP64) ? run_persistent<G, double>(st, p, prm, result, net_corr, stream)
                                    : run_persistent<G, float>(st, p, prm, result, net_corr, stream);
        if (s != MCD_OK) return s;
        if (prm->mode == MCD_MIXED && result != MCD_OK && result != MCD_ETIMEOUT) {
            // the FP32 recursion failed (diverged or broke down): finish in
            // FP64 from the last folded iterate, which the failed cycle
            // never touched
            const Scalars &hm = *w->h_sc;
            mixed_iters = hm.iter;
            mixed_div = hm.divergences;
            mixed_upd = hm.updates;
            fallback = (result == MCD_ENOCONV) ? 6 : (hm.diverged > 0 ? hm.diverged : 7);
            Scalars re;
            memset(&re, 0, sizeof(re));
            re.max_iter = std::max(1, init.max_iter - hm.iter);
            re.unknowns = hm.unknowns;
            MCD_CUDA_TRY(cudaMemcpyAsync(w->sc, &re, sizeof(re), cudaMemcpyHostToDevice, stream));
            s = ensure_workspace(const_cast<mcd_stencils *>(st), MCD_FP64);
            if (s != MCD_OK) return s;
            s = run_persistent<G, double>(st, p, prm, result, net_corr, stream);
            if (s != MCD_OK) return s;
        }
    } else if (prm->mode == MCD_FP64) {
        for (;; ++outer) {
            // FP64 residual of the current iterate (primes the Krylov scalars)
            s = residual<G>(st, p, prm->tol, 1, stream);
            if (s != MCD_OK) return s;
            s = read_scalars(w, stream);
            if (s != MCD_OK) return s;
            const Scalars &h = *w->h_sc;
            if (h.done == 4) { result = MCD_ENONFINITE; break; }
            if (h.done == 1) { result = MCD_OK; break; }
            if (h.iter >= init.max_iter) { result = MCD_ENOCONV; break; }
            if (outer >= max_outer) { result = MCD_ENOCONV; break; }
            Vecs<double> vv{p, w->r64, w->drh, {w->dp[0], w->dp[1]}, {w->dv[0], w->dv[1]}, w->ds, w->dt};
            s = run_krylov<G, double, double>(st, st->row64, vv, check_every, 1e-14, max_launch, stream);
            if (s != MCD_OK) return s;
            const int done = w->h_sc->done;
            if (done == 4) { result = MCD_ENONFINITE; break; }
            if (done == 3) { result = MCD_EBREAKDOWN; break; }
            // done 1 (recursive residual converged) or 2 (max_iter): the next
            // FP64 residual decides, and restarts the recurrence if needed
        }
    } else {
        s = run_mixed<G>(st, p, prm, check_every, max_launch, outer, result, stream);
        if (s != MCD_OK) return s;
    }
    // Block lower-triangular system: no inner row references a Neumann DP
    // (Eq. (16) leaves Gamma_N out of Lambda_c), so the Krylov solve above ran
    // on the interior block with the Neumann rows held fixed.  Their values
    // now follow from their own rows; then the full FP64 residual decides.
    if (result == MCD_OK && st->has_neumann) {
        // Jacobi sweeps on the Neumann rows converge geometrically; the
        // interior block may have stopped just below tol, leaving them a thin
        // margin, so the rounds grow (8, 8, 16, 16, ... 256: about 1000
        // sweeps at most) until the full residual meets tol
        result = MCD_ENOCONV;
        for (int round = 0; round < 12; ++round) {
            s = neumann_sweeps<G>(st, p, 8 << (round / 2), stream);
            if (s != MCD_OK) return s;
            s = residual<G>(st, p, prm->tol, 0, stream);
            if (s != MCD_OK) return s;
            s = read_scalars(w, stream);
            if (s != MCD_OK) return s;
            if (w->h_sc->done == 4) { result = MCD_ENONFINITE; break; }
            if (w->h_sc->done == 1) { result = MCD_OK; break; }
        }
    }
    if (result == MCD_OK && prm->net && prm->net_dprev) {
        s = net_store_increment(prm->net, st, p, prm->net_dprev, stream);
        if (s != MCD_OK) return s;
    }
    const Scalars &h = *w->h_sc;
    if (info) {
        info->iters = h.iter + mixed_iters;
        info->refinements = outer;
        info->fallback = fallback;
        info->net_corrections = net_corr;
        info->discarded = mixed_div + h.divergences;
        if (prm->check_every >= 0) info->refinements = mixed_upd + h.updates;
        info->restarts = h.restarts;
        info->b_norm = sqrt(h.bb64);
        info->rel_res = h.bb64 > 0.0 ? sqrt(h.rr64 / h.bb64) : 0.0;
        info->unknowns = (int64_t)h.unknowns;
        info->rel_res_guess = -1.0;
        info->rel_res_start = -1.0;
        if (prm->net && ws_sc[4] > 0.0) {
            info->rel_res_guess = sqrt(ws_sc[3] / ws_sc[4]);
            info->rel_res_start = sqrt(ws_sc[6] / ws_sc[4]);
        }
    }
    if (result == MCD_ENOCONV) set_error("solve reached max_iter / max_refine before tol");
    if (result == MCD_ENONFINITE) set_error("non-finite value in right-hand side or residual");
    if (result == MCD_EBREAKDOWN || result == MCD_ENONFINITE) {
        char buf[512];
        snprintf(buf, sizeof(buf),
                 "%s (iter %d, refinement %d, restarts %d, rho %.3e, r^.v %.3e, t.s %.3e, t.t %.3e, "
                 "s.s %.3e, r.r %.3e, tol2 %.3e, ||r64||^2 %.3e, ||b||^2 %.3e)",
                 result == MCD_EBREAKDOWN ? "Bi-CGSTAB breakdown" : "non-finite value", h.iter, outer,
                 h.restarts, h.rho, h.rv, h.ts, h.tt, h.ss, h.rr, h.tol2, h.rr64, h.bb64);
        set_error(buf);
    }
    return result;
}

}  // namespace mcd

using namespace mcd;

extern "C" mcd_status mcd_solver_set_staging(int on) {
    g_no_stage = on ? 0 : 1;
    return MCD_OK;
}

extern "C" mcd_status mcd_trace_enable(int on) {
    if (on && !g_trace) {
        MCD_CUDA_TRY(cudaMalloc(&g_trace, (512 + 6144 + 2048) * sizeof(unsigned long long)));
        MCD_CUDA_TRY(cudaMemset(g_trace, 0, (512 + 6144 + 2048) * sizeof(unsigned long long)));
    } else if (!on && g_trace) {
        cudaFree(g_trace);
        g_trace = nullptr;
    }
    return MCD_OK;
}

extern "C" mcd_status mcd_trace_read(unsigned long long *host_out) {
    MCD_CHECK_ARG(host_out, "NULL argument");
    MCD_CHECK_ARG(g_trace, "tracing is not enabled");
    MCD_CUDA_TRY(cudaMemcpy(host_out, g_trace, (512 + 6144 + 2048) * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return MCD_OK;
}

extern "C" mcd_status mcd_solve_pressure(const mcd_stencils *st, const double *rhs_dev,
                                         const double *bnd_dev, double *p_dev,
                                         const mcd_solve_params *prm, mcd_solve_info *info,
                                         mcd_stream_t stream) {
    MCD_CHECK_ARG(st && rhs_dev && bnd_dev && p_dev && prm, "NULL argument");
    MCD_CHECK_ARG(prm->tol > 0.0, "tol must be positive");
    MCD_CHECK_ARG(prm->mode == MCD_FP64 || prm->mode == MCD_MIXED, "unknown mode");
    MCD_CHECK_ARG(prm->mode != MCD_MIXED || st->row32, "MIXED solve needs an MCD_MIXED stencil handle");
    MCD_CHECK_ARG(prm->mode != MCD_MIXED || (prm->inner_tol > 0.0 && prm->inner_tol < 1.0),
                  "inner_tol must be in (0, 1)");
    MCD_CHECK_ARG(!prm->precond || (prm->mode == MCD_MIXED && prm->barriers != 3 && prm->check_every >= 0),
                  "a preconditioner network needs a MIXED solve on the one- or two-barrier persistent schedule");
    mcd_status s = mcd_stencils_check(st, nullptr, stream);
    if (s != MCD_OK) return s;
    s = ensure_workspace(const_cast<mcd_stencils *>(st), prm->mode);
    if (s != MCD_OK) return s;
    if (st->shape == 2) return solve_impl<2>(st, rhs_dev, bnd_dev, p_dev, prm, info, stream);
    if (st->shape == 3) return solve_impl<3>(st, rhs_dev, bnd_dev, p_dev, prm, info, stream);
    return solve_impl<9>(st, rhs_dev, bnd_dev, p_dev, prm, info, stream);
}

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
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mcd {

struct Scalars {
    double rho, alpha, omega, beta;
    double rhat2;     // ||r^||^2 (breakdown test)
    double tol2;      // squared absolute tolerance on the recursive residual
    double rr, ss, ts, tt, rv;
    double rr64, bb64;  // last FP64 residual: ||b - A x||^2, ||b||^2
    int iter, max_iter;
    int done;         // 0 running, 1 converged, 2 max_iter, 3 breakdown, 4 nonfinite
    int restart;      // next KA sets r^ = r and p = r
    int restarts;
    int s_conv;       // ||s|| small: KC does x += alpha p and stops
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
    double *partials = nullptr;  // [4][max(nblk, nblk1)]
    unsigned int *counter = nullptr;
    Scalars *sc = nullptr;
    Scalars *h_sc = nullptr;     // pinned host mirror
    int pstride = 0;
};

void free_workspace(mcd_stencils *st) {
    Workspace *w = st->ws;
    if (!w) return;
    cudaFree(w->b); cudaFree(w->r64);
    cudaFree(w->dr); cudaFree(w->drh); cudaFree(w->dp[0]); cudaFree(w->dp[1]);
    cudaFree(w->dv[0]); cudaFree(w->dv[1]); cudaFree(w->ds); cudaFree(w->dt);
    cudaFree(w->fr); cudaFree(w->frh); cudaFree(w->fp[0]); cudaFree(w->fp[1]);
    cudaFree(w->fv[0]); cudaFree(w->fv[1]); cudaFree(w->fs); cudaFree(w->ft); cudaFree(w->fd);
    cudaFree(w->partials); cudaFree(w->counter); cudaFree(w->sc);
    cudaFreeHost(w->h_sc);
    delete w;
    st->ws = nullptr;
}

// Tile shape per dimension (one DP per thread, 256 threads).
template <int DIM> struct Tile;
template <> struct Tile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<3> { static constexpr int X = 32, Y = 4, Z = 2; };

template <int DIM> struct HaloDims {
    static constexpr int HX = Tile<DIM>::X + 2;
    static constexpr int HY = Tile<DIM>::Y + 2;
    static constexpr int HZ = (DIM == 3) ? Tile<DIM>::Z + 2 : 1;
    static constexpr int H = HX * HY * HZ;
    static constexpr int S = (DIM == 2) ? 9 : 27;
};

__device__ __forceinline__ int wrap_clamp(int v, int n, int per) {
    if (v < 0) return per ? v + n : 0;
    if (v >= n) return per ? v - n : n - 1;
    return v;
}

// Deterministic block reduction of NV values; thread 0 writes them to
// partials[q * stride + block].
template <int NV, typename A>
__device__ __forceinline__ void block_partials(A (&v)[NV], double *partials, int stride, int block) {
    __shared__ double wsum[NV][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if ((tid & 31) == 0)
        for (int q = 0; q < NV; ++q) wsum[q][tid >> 5] = (double)v[q];
    __syncthreads();
    if (tid < 32) {
        const int nw = nthreads >> 5;
        for (int q = 0; q < NV; ++q) {
            double x = (tid < nw) ? wsum[q][tid] : 0.0;
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (tid == 0) partials[q * stride + block] = x;
        }
    }
}

// Returns true in the block that arrives last; that block then holds the
// totals of the NV partial sums in out[] (valid in every thread).
template <int NV>
__device__ __forceinline__ bool last_block_totals(const double *partials, int stride, int nblocks,
                                                  unsigned int *counter, double (&out)[NV]) {
    __shared__ bool is_last;
    __shared__ double red[NV][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        is_last = (t == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    for (int q = 0; q < NV; ++q) {
        double acc = 0.0;
        for (int b = tid; b < nblocks; b += nthreads) acc += __ldcg(partials + q * stride + b);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) red[q][tid >> 5] = acc;
    }
    __syncthreads();
    for (int q = 0; q < NV; ++q) {
        double x = 0.0;
        for (int w = 0; w < (nthreads >> 5); ++w) x += red[q][w];
        out[q] = x;
    }
    if (tid == 0) *counter = 0u;
    return true;
}

struct TileArgs {
    Geo g;
    int bx, by, bz;      // tiles per axis
};

template <int DIM>
__device__ __forceinline__ void tile_origin(const TileArgs &ta, int &x0, int &y0, int &z0, int &blk) {
    blk = blockIdx.x;
    const int tx = blk % ta.bx;
    const int rest = blk / ta.bx;
    const int ty = rest % ta.by;
    const int tz = rest / ta.by;
    x0 = tx * Tile<DIM>::X;
    y0 = ty * Tile<DIM>::Y;
    z0 = tz * Tile<DIM>::Z;
}

// Global index of halo element h of the tile at (x0, y0, z0).
template <int DIM>
__device__ __forceinline__ int64_t halo_index(const Geo &g, int h, int x0, int y0, int z0) {
    using HD = HaloDims<DIM>;
    const int hx = h % HD::HX;
    const int hy = (h / HD::HX) % HD::HY;
    const int hz = h / (HD::HX * HD::HY);
    const int gx = wrap_clamp(x0 + hx - 1, g.n[0], g.per[0]);
    const int gy = wrap_clamp(y0 + hy - 1, g.n[1], g.per[1]);
    if (DIM == 2) return (int64_t)gx + (int64_t)g.n[0] * gy;
    const int gz = wrap_clamp(z0 + hz - 1, g.n[2], g.per[2]);
    return (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
}

// sum_s row[s][k] * tile[neighbour s] for the thread's own DP.
template <int DIM, typename T>
__device__ __forceinline__ T stencil_from_tile(const T *__restrict__ row, int64_t N, int64_t k,
                                               const T *tile, int lx, int ly, int lz) {
    using HD = HaloDims<DIM>;
    T acc = 0;
#pragma unroll
    for (int s = 0; s < HD::S; ++s) {
        const int ox = s % 3, oy = (s / 3) % 3, oz = s / 9;
        const int h = (lx + ox) + HD::HX * ((ly + oy) + HD::HY * (lz + oz));
        acc += row[(int64_t)s * N + k] * tile[h];
    }
    return acc;
}

// ---- KA: p = r + beta (p_old - omega v_old); v = A p; partial r^.v -------
template <int DIM, typename T, typename A>
__global__ void __launch_bounds__(256) bicg_ka(TileArgs ta, const T *__restrict__ row, const T *__restrict__ r,
                                               T *__restrict__ rhat, const T *__restrict__ p_old,
                                               const T *__restrict__ v_old, T *__restrict__ p_new,
                                               T *__restrict__ v_new, Scalars *sc, double *partials,
                                               int pstride, unsigned int *counter) {
    using HD = HaloDims<DIM>;
    __shared__ T tile[HD::H];
    if (sc->done) return;
    const T beta = (T)sc->beta, omega = (T)sc->omega;
    const int restart = sc->restart;
    int x0, y0, z0, blk;
    tile_origin<DIM>(ta, x0, y0, z0, blk);
    const Geo &g = ta.g;
    const int tid = threadIdx.x;
    for (int h = tid; h < HD::H; h += 256) {
        const int64_t j = halo_index<DIM>(g, h, x0, y0, z0);
        const T rj = r[j];
        tile[h] = restart ? rj : rj + beta * (p_old[j] - omega * v_old[j]);
    }
    __syncthreads();
    const int lx = tid % Tile<DIM>::X;
    const int ly = (tid / Tile<DIM>::X) % Tile<DIM>::Y;
    const int lz = tid / (Tile<DIM>::X * Tile<DIM>::Y);
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    A dot[1] = {0};
    if (gx < g.n[0] && gy < g.n[1] && (DIM == 2 || gz < g.n[2])) {
        const int64_t k = (DIM == 2) ? (int64_t)gx + (int64_t)g.n[0] * gy
                                     : (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
        const int hc = (lx + 1) + HD::HX * ((ly + 1) + HD::HY * (DIM == 3 ? lz + 1 : 0));
        const T pk = tile[hc];
        p_new[k] = pk;
        T rh;
        if (restart) { rh = r[k]; rhat[k] = rh; } else { rh = rhat[k]; }
        const T vk = stencil_from_tile<DIM, T>(row, g.N, k, tile, lx, ly, lz);
        v_new[k] = vk;
        dot[0] = (A)rh * (A)vk;
    }
    block_partials<1, A>(dot, partials, pstride, blk);
    double tot[1];
    if (last_block_totals<1>(partials, pstride, gridDim.x, counter, tot) && tid == 0) {
        sc->rv = tot[0];
        sc->restart = 0;
        const double alpha = sc->rho / tot[0];
        if (!isfinite(alpha)) { sc->done = 3; return; }
        sc->alpha = alpha;
    }
}

// ---- KB: s = r - alpha v; t = A s; partials t.s, t.t, s.s ------------------
template <int DIM, typename T, typename A>
__global__ void __launch_bounds__(256) bicg_kb(TileArgs ta, const T *__restrict__ row, const T *__restrict__ r,
                                               const T *__restrict__ v, T *__restrict__ s_out,
                                               T *__restrict__ t_out, Scalars *sc, double *partials,
                                               int pstride, unsigned int *counter) {
    using HD = HaloDims<DIM>;
    __shared__ T tile[HD::H];
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    int x0, y0, z0, blk;
    tile_origin<DIM>(ta, x0, y0, z0, blk);
    const Geo &g = ta.g;
    const int tid = threadIdx.x;
    for (int h = tid; h < HD::H; h += 256) {
        const int64_t j = halo_index<DIM>(g, h, x0, y0, z0);
        tile[h] = r[j] - alpha * v[j];
    }
    __syncthreads();
    const int lx = tid % Tile<DIM>::X;
    const int ly = (tid / Tile<DIM>::X) % Tile<DIM>::Y;
    const int lz = tid / (Tile<DIM>::X * Tile<DIM>::Y);
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    A dot[3] = {0, 0, 0};
    if (gx < g.n[0] && gy < g.n[1] && (DIM == 2 || gz < g.n[2])) {
        const int64_t k = (DIM == 2) ? (int64_t)gx + (int64_t)g.n[0] * gy
                                     : (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
        const int hc = (lx + 1) + HD::HX * ((ly + 1) + HD::HY * (DIM == 3 ? lz + 1 : 0));
        const T sk = tile[hc];
        s_out[k] = sk;
        const T tk = stencil_from_tile<DIM, T>(row, g.N, k, tile, lx, ly, lz);
        t_out[k] = tk;
        dot[0] = (A)tk * (A)sk;
        dot[1] = (A)tk * (A)tk;
        dot[2] = (A)sk * (A)sk;
    }
    block_partials<3, A>(dot, partials, pstride, blk);
    double tot[3];
    if (last_block_totals<3>(partials, pstride, gridDim.x, counter, tot) && tid == 0) {
        sc->ts = tot[0];
        sc->tt = tot[1];
        sc->ss = tot[2];
        if (!isfinite(tot[0] + tot[1] + tot[2])) { sc->done = 4; return; }
        if (tot[2] <= sc->tol2) { sc->s_conv = 1; return; }
        if (tot[1] == 0.0) { sc->done = 3; return; }
        sc->omega = tot[0] / tot[1];
    }
}

// ---- KC: x += alpha p + omega s; r = s - omega t; partials r^.r, r.r -------
template <typename T, typename A>
__global__ void __launch_bounds__(256) bicg_kc(int64_t N, T *__restrict__ x, T *__restrict__ r,
                                               const T *__restrict__ rhat, const T *__restrict__ p,
                                               const T *__restrict__ s, const T *__restrict__ t,
                                               Scalars *sc, double *partials, int pstride,
                                               unsigned int *counter, double eps_breakdown) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha, omega = (T)sc->omega;
    const int sconv = sc->s_conv;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    A dot[2] = {0, 0};
    if (k < N) {
        const T sk = s[k];
        T rk;
        if (sconv) {
            x[k] += alpha * p[k];
            rk = sk;
        } else {
            x[k] += alpha * p[k] + omega * sk;
            rk = sk - omega * t[k];
        }
        r[k] = rk;
        dot[0] = (A)rhat[k] * (A)rk;
        dot[1] = (A)rk * (A)rk;
    }
    block_partials<2, A>(dot, partials, pstride, blockIdx.x);
    double tot[2];
    if (last_block_totals<2>(partials, pstride, gridDim.x, counter, tot) && threadIdx.x == 0) {
        const double rho_new = tot[0], rr = tot[1];
        sc->rr = rr;
        sc->iter += 1;
        if (!isfinite(rho_new + rr)) { sc->done = 4; return; }
        if (sconv || rr <= sc->tol2) { sc->done = 1; return; }
        if (sc->iter >= sc->max_iter) { sc->done = 2; return; }
        if (fabs(rho_new) <= eps_breakdown * sqrt(sc->rhat2 * rr)) {
            sc->restarts += 1;
            if (sc->restarts > 50) { sc->done = 3; return; }
            sc->restart = 1;
            sc->rho = rr;
            sc->rhat2 = rr;
            sc->beta = 0.0;
            return;
        }
        sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
        sc->rho = rho_new;
    }
}

// ---- FP64 residual r = b - A x (1D; neighbours through L1) ---------------
// Its last block records ||r||^2, ||b||^2 and primes the Krylov scalars for a
// (re)start from this residual with tolerance tol2 = (tol ||b||)^2.
template <int DIM>
__global__ void __launch_bounds__(256) residual64(Geo g, const double *__restrict__ row, const double *__restrict__ b,
                                                  const double *__restrict__ x, double *__restrict__ r,
                                                  Scalars *sc, double *partials, int pstride,
                                                  unsigned int *counter, double tol) {
    constexpr int S = (DIM == 2) ? 9 : 27;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dot[2] = {0.0, 0.0};
    if (k < N) {
        int c[3] = {0, 0, 0};
        c[0] = (int)(k % g.n[0]);
        const int64_t rest = k / g.n[0];
        if (DIM == 2) c[1] = (int)rest; else { c[1] = (int)(rest % g.n[1]); c[2] = (int)(rest / g.n[1]); }
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = s / 9 - 1;
            const int gx = wrap_clamp(c[0] + ox, g.n[0], g.per[0]);
            const int gy = wrap_clamp(c[1] + oy, g.n[1], g.per[1]);
            int64_t j = (int64_t)gx + (int64_t)g.n[0] * gy;
            if (DIM == 3) {
                const int gz = wrap_clamp(c[2] + oz, g.n[2], g.per[2]);
                j = (int64_t)gx + (int64_t)g.n[0] * ((int64_t)gy + (int64_t)g.n[1] * gz);
            }
            acc += row[(int64_t)s * N + k] * x[j];
        }
        const double bk = b[k];
        const double rk = bk - acc;
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
        sc->tol2 = tol * tol * tot[1];
        if (!isfinite(tot[0] + tot[1])) sc->done = 4;
        else sc->done = (tot[0] <= sc->tol2) ? 1 : 0;
    }
}

// r32 = (float) r64, d = 0; primes the FP32 inner solve with relative
// tolerance inner_tol on ||r32||.
__global__ void __launch_bounds__(256) prep_inner(int64_t N, const double *__restrict__ r64, float *__restrict__ r32,
                                                  float *__restrict__ d, Scalars *sc, double *partials,
                                                  int pstride, unsigned int *counter, double inner_tol) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dot[1] = {0.0f};
    if (k < N) {
        const float rk = (float)r64[k];
        r32[k] = rk;
        d[k] = 0.0f;
        dot[0] = rk * rk;
    }
    block_partials<1, float>(dot, partials, pstride, blockIdx.x);
    double tot[1];
    if (last_block_totals<1>(partials, pstride, gridDim.x, counter, tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        sc->rho = tot[0];
        sc->rhat2 = tot[0];
        sc->beta = 0.0;
        sc->alpha = 1.0;
        sc->omega = 1.0;
        sc->restart = 1;
        sc->s_conv = 0;
        sc->tol2 = inner_tol * inner_tol * tot[0];
        sc->done = (tot[0] == 0.0) ? 1 : 0;
    }
}

__global__ void add_correction(int64_t N, double *__restrict__ x, const float *__restrict__ d) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) x[k] += (double)d[k];
}

// Dirichlet entries of the guess take their value (b = g there); void = 0.
__global__ void fix_guess(int64_t N, const int8_t *__restrict__ kind, const double *__restrict__ b,
                          double *__restrict__ x) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int8_t kd = kind[k];
    if (kd == KIND_DIRICHLET) x[k] = b[k];
    else if (kd == KIND_VOID) x[k] = 0.0;
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
        chk(cudaMalloc(&w->partials, 4 * (size_t)w->pstride * sizeof(double)));
        chk(cudaMalloc(&w->counter, sizeof(unsigned int)));
        chk(cudaMalloc(&w->sc, sizeof(Scalars)));
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

// Launch `count` Bi-CGSTAB iterations (3 kernels each); parity selects the
// p / v ping-pong buffers and is advanced.
template <int DIM, typename T, typename A>
static mcd_status launch_iters(const mcd_stencils *st, const T *row, Vecs<T> &vv, int &parity,
                               int count, double eps_breakdown, cudaStream_t stream) {
    Workspace *w = st->ws;
    const Geo &g = st->geo;
    TileArgs ta;
    ta.g = g;
    ta.bx = (g.n[0] + Tile<DIM>::X - 1) / Tile<DIM>::X;
    ta.by = (g.n[1] + Tile<DIM>::Y - 1) / Tile<DIM>::Y;
    ta.bz = (DIM == 3) ? (g.n[2] + Tile<DIM>::Z - 1) / Tile<DIM>::Z : 1;
    for (int it = 0; it < count; ++it) {
        const int a = parity, b = parity ^ 1;
        bicg_ka<DIM, T, A><<<w->nblk, 256, 0, stream>>>(ta, row, vv.r, vv.rh, vv.p[a], vv.v[a], vv.p[b],
                                                        vv.v[b], w->sc, w->partials, w->pstride, w->counter);
        bicg_kb<DIM, T, A><<<w->nblk, 256, 0, stream>>>(ta, row, vv.r, vv.v[b], vv.s, vv.t, w->sc,
                                                        w->partials, w->pstride, w->counter);
        bicg_kc<T, A><<<w->nblk1, 256, 0, stream>>>(g.N, vv.x, vv.r, vv.rh, vv.p[b], vv.s, vv.t, w->sc,
                                                    w->partials, w->pstride, w->counter, eps_breakdown);
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
template <int DIM, typename T, typename A>
static mcd_status run_krylov(const mcd_stencils *st, const T *row, Vecs<T> &vv, int check_every,
                             double eps_breakdown, int max_launch, cudaStream_t stream) {
    Workspace *w = st->ws;
    int parity = 0;
    int chunk = 4;
    int launched = 0;
    for (;;) {
        mcd_status s = launch_iters<DIM, T, A>(st, row, vv, parity, chunk, eps_breakdown, stream);
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

template <int DIM>
static mcd_status residual(const mcd_stencils *st, const double *x, double tol, cudaStream_t stream) {
    Workspace *w = st->ws;
    residual64<DIM><<<w->nblk1, 256, 0, stream>>>(st->geo, st->row64, w->b, x, w->r64, w->sc, w->partials,
                                                  w->pstride, w->counter, tol);
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

template <int DIM>
static mcd_status solve_impl(const mcd_stencils *st, const double *rhs, const double *bnd, double *p,
                             const mcd_solve_params *prm, mcd_solve_info *info, cudaStream_t stream) {
    Workspace *w = st->ws;
    const int64_t N = st->geo.N;
    mcd_status s = mcd_assemble_rhs(st, rhs, bnd, w->b, stream);
    if (s != MCD_OK) return s;
    fix_guess<<<w->nblk1, 256, 0, stream>>>(N, st->kind, w->b, p);
    MCD_LAUNCH_CHECK();

    Scalars init;
    memset(&init, 0, sizeof(init));
    init.max_iter = prm->max_iter > 0 ? prm->max_iter : 1 << 30;
    MCD_CUDA_TRY(cudaMemcpyAsync(w->sc, &init, sizeof(init), cudaMemcpyHostToDevice, stream));
    const int check_every = prm->check_every > 0 ? prm->check_every : 64;
    const int max_outer = prm->max_refine > 0 ? prm->max_refine : 50;
    const int max_launch = (init.max_iter > (1 << 29) ? (1 << 29) : init.max_iter) + 2 * check_every;

    mcd_status result = MCD_ENOCONV;
    int outer = 0;
    for (;; ++outer) {
        // FP64 residual of the current iterate (primes the Krylov scalars)
        s = residual<DIM>(st, p, prm->tol, stream);
        if (s != MCD_OK) return s;
        s = read_scalars(w, stream);
        if (s != MCD_OK) return s;
        const Scalars &h = *w->h_sc;
        if (h.done == 4) { result = MCD_ENONFINITE; break; }
        if (h.done == 1) { result = MCD_OK; break; }
        if (h.iter >= init.max_iter) { result = MCD_ENOCONV; break; }
        if (outer >= max_outer) { result = MCD_ENOCONV; break; }
        if (prm->mode == MCD_FP64) {
            Vecs<double> vv{p, w->r64, w->drh, {w->dp[0], w->dp[1]}, {w->dv[0], w->dv[1]}, w->ds, w->dt};
            s = run_krylov<DIM, double, double>(st, st->row64, vv, check_every, 1e-14, max_launch, stream);
        } else {
            prep_inner<<<w->nblk1, 256, 0, stream>>>(N, w->r64, w->fr, w->fd, w->sc, w->partials, w->pstride,
                                                     w->counter, prm->inner_tol);
            MCD_LAUNCH_CHECK();
            Vecs<float> vv{w->fd, w->fr, w->frh, {w->fp[0], w->fp[1]}, {w->fv[0], w->fv[1]}, w->fs, w->ft};
            s = run_krylov<DIM, float, float>(st, st->row32, vv, check_every, 1e-7, max_launch, stream);
            if (s == MCD_OK) {
                add_correction<<<w->nblk1, 256, 0, stream>>>(N, p, w->fd);
                MCD_LAUNCH_CHECK();
            }
        }
        if (s != MCD_OK) return s;
        const int done = w->h_sc->done;
        if (done == 4) { result = MCD_ENONFINITE; break; }
        if (done == 3) { result = MCD_EBREAKDOWN; break; }
        // done 1 (inner converged) or 2 (max_iter): re-check with FP64 residual
        // clear the inner status so the next residual can prime a restart
        int zero = 0;
        MCD_CUDA_TRY(cudaMemcpyAsync(&w->sc->done, &zero, sizeof(int), cudaMemcpyHostToDevice, stream));
    }
    const Scalars &h = *w->h_sc;
    if (info) {
        info->iters = h.iter;
        info->refinements = outer;
        info->restarts = h.restarts;
        info->b_norm = sqrt(h.bb64);
        info->rel_res = h.bb64 > 0.0 ? sqrt(h.rr64 / h.bb64) : 0.0;
    }
    if (result == MCD_ENOCONV) set_error("solve reached max_iter / max_refine before tol");
    if (result == MCD_ENONFINITE) set_error("non-finite value in right-hand side or residual");
    if (result == MCD_EBREAKDOWN) set_error("Bi-CGSTAB breakdown");
    return result;
}

}  // namespace mcd

using namespace mcd;

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
    MCD_CHECK_ARG(prm->net == nullptr, "network warm start is not available in this build");
    mcd_status s = mcd_stencils_check(st, nullptr, stream);
    if (s != MCD_OK) return s;
    s = ensure_workspace(const_cast<mcd_stencils *>(st), prm->mode);
    if (s != MCD_OK) return s;
    if (st->mesh.dim == 2) return solve_impl<2>(st, rhs_dev, bnd_dev, p_dev, prm, info, stream);
    return solve_impl<3>(st, rhs_dev, bnd_dev, p_dev, prm, info, stream);
}

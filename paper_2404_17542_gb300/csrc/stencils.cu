// MLS stencil weights and the pressure-Poisson rows (arXiv 2404.17542,
// Sec. 3.2, Eqs. (12)-(17); Sec. 3.3, Eq. (21), (23)).
//
// One thread per DP.  Pass 1 gathers the DP's 3x3 (3x3x3, or expanded 9x9)
// cells, forms the
// moment matrix M = sum w p p^T (+ Neumann terms w p^N p^N^T) and the vector
// sum w p, and factors M by Cholesky in registers.  Pass 2 revisits the
// neighbours and writes, slot by slot, z = M^{-1} (w p) -- the weight that
// neighbour carries in every derivative -- into slot-major SoA arrays, so a
// warp's stores for one slot are contiguous.  The centre weight is
// -M^{-1} sum_j w_j p_j, known before pass 2, which lets Neumann rows be
// scaled (row equilibration) without buffering the row.
//
// FP64 throughout: the FP64 rows are the matrix the refinement residual is
// judged on; the FP32 copy used by the inner Krylov solve is their rounding.
#include <cuda.h>
#include <math.h>

#include <string.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace mcd {

template <int DIM> struct Basis;

template <> struct Basis<2> {
    static constexpr int NB = 5;
    static constexpr int S = 9;
    // p(X) = (X, Y, X^2/2, XY, Y^2/2)  (Eq. (13))
    __device__ static void value(const double *X, double *p) {
        p[0] = X[0]; p[1] = X[1];
        p[2] = 0.5 * X[0] * X[0]; p[3] = X[0] * X[1]; p[4] = 0.5 * X[1] * X[1];
    }
    // p^N = n . grad_X p(X)  (Neumann term of Eq. (15))
    __device__ static void normal(const double *X, const double *n, double *p) {
        p[0] = n[0]; p[1] = n[1];
        p[2] = n[0] * X[0]; p[3] = n[0] * X[1] + n[1] * X[0]; p[4] = n[1] * X[1];
    }
    __device__ static int order(int c) { return c < 2 ? 1 : 2; }
    __device__ static bool is_lap(int c) { return c == 2 || c == 4; }
};

template <> struct Basis<3> {
    static constexpr int NB = 9;
    static constexpr int S = 27;
    // (X, Y, Z, X^2/2, Y^2/2, Z^2/2, XY, YZ, XZ)
    __device__ static void value(const double *X, double *p) {
        p[0] = X[0]; p[1] = X[1]; p[2] = X[2];
        p[3] = 0.5 * X[0] * X[0]; p[4] = 0.5 * X[1] * X[1]; p[5] = 0.5 * X[2] * X[2];
        p[6] = X[0] * X[1]; p[7] = X[1] * X[2]; p[8] = X[0] * X[2];
    }
    __device__ static void normal(const double *X, const double *n, double *p) {
        p[0] = n[0]; p[1] = n[1]; p[2] = n[2];
        p[3] = n[0] * X[0]; p[4] = n[1] * X[1]; p[5] = n[2] * X[2];
        p[6] = n[0] * X[1] + n[1] * X[0];
        p[7] = n[1] * X[2] + n[2] * X[1];
        p[8] = n[0] * X[2] + n[2] * X[0];
    }
    __device__ static int order(int c) { return c < 3 ? 1 : 2; }
    __device__ static bool is_lap(int c) { return c >= 3 && c <= 5; }
};

struct BuildArgs {
    Geo g;
    const double *pos;
    const int8_t *mask;
    const double *normal;
    uint8_t bc[128];
    int weight_kind;
    double r_e, r_s;
    double *row64;
    float *row32;
    double *ql64;
    double *d64;
    double *qd64;
    double *rscale;
    int8_t *kind;
    unsigned long long *bad;
};

__device__ __forceinline__ double mls_weight(double r, int kind, double r_e) {
    if (kind == MCD_W_COS2) {
        if (r > r_e) return 0.0;
        double c = cos(M_PI * r / (2.0 * r_e));
        return c * c;
    }
    if (kind == MCD_W_LSMPS) {
        if (!(r < r_e)) return 0.0;
        const double q = 1.0 - r / r_e;
        return q * q;
    }
    double q = r / r_e;
    return exp(-q * q);
}

// Packed lower-triangular index of (a, b), a >= b.
__device__ __forceinline__ int tri(int a, int b) { return a * (a + 1) / 2 + b; }

// In-place Cholesky of the packed matrix (first nf rows); false if a pivot is
// not positive (the matrix is not positive definite) or not finite.
template <int NB>
__device__ bool cholesky(double *L, int nf) {
    for (int j = 0; j < NB; ++j) {
        if (j >= nf) break;
        double d = L[tri(j, j)];
        for (int k = 0; k < j; ++k) d -= L[tri(j, k)] * L[tri(j, k)];
        if (!(d > 0.0) || !isfinite(d)) return false;
        d = sqrt(d);
        L[tri(j, j)] = d;
        double inv = 1.0 / d;
        for (int i = j + 1; i < NB; ++i) {
            if (i >= nf) break;
            double v = L[tri(i, j)];
            for (int k = 0; k < j; ++k) v -= L[tri(i, k)] * L[tri(j, k)];
            L[tri(i, j)] = v * inv;
        }
    }
    return true;
}

// Solve (L L^T) z = b in place (first nf entries).
template <int NB>
__device__ void chol_solve(const double *L, int nf, double *z) {
    for (int i = 0; i < NB; ++i) {
        if (i >= nf) break;
        double v = z[i];
        for (int k = 0; k < i; ++k) v -= L[tri(i, k)] * z[k];
        z[i] = v / L[tri(i, i)];
    }
    for (int i = NB - 1; i >= 0; --i) {
        if (i >= nf) continue;
        double v = z[i];
        for (int k = i + 1; k < NB; ++k) {
            if (k >= nf) break;
            v -= L[tri(k, i)] * z[k];
        }
        z[i] = v / L[tri(i, i)];
    }
}

template <int DIM>
struct Nbr {
    int64_t j;
    bool valid;
    double shift[DIM];
};

template <int DIM>
__device__ __forceinline__ void decode(const Geo &g, int64_t k, int *c) {
    c[0] = (int)(k % g.n[0]);
    int64_t rest = k / g.n[0];
    if (DIM == 2) {
        c[1] = (int)rest;
    } else {
        c[1] = (int)(rest % g.n[1]);
        c[2] = (int)(rest / g.n[1]);
    }
}

template <int G, int DIM = Shape<G>::dim>
__device__ __forceinline__ Nbr<DIM> neighbour(const Geo &g, const int *c, int s) {
    Nbr<DIM> r;
    r.valid = true;
    int o[3];
    slot_offset<G>(s, o);
    int v[3];
    for (int d = 0; d < DIM; ++d) {
        double sh;
        v[d] = nb_coord(c[d], o[d], g.n[d], g.per[d], g.len[d], sh, r.valid);
        r.shift[d] = sh;
    }
    r.j = (DIM == 2) ? (int64_t)v[0] + (int64_t)g.n[0] * v[1]
                     : (int64_t)v[0] + (int64_t)g.n[0] * ((int64_t)v[1] + (int64_t)g.n[1] * v[2]);
    return r;
}

// Weights of DP k of the system with geometry g whose arrays start at DP
// offset `off` in the arrays of `a` (a batch of systems stored back to back,
// each in its own [slot][N] layout; off = 0 for a single system).
template <int G>
__device__ __forceinline__ void build_dp(const BuildArgs &a, const Geo &g, int64_t off, int64_t k,
                                         double r_e, double r_s) {
    constexpr int DIM = Shape<G>::dim;
    using B = Basis<DIM>;
    constexpr int NB = B::NB;
    constexpr int S = Shape<G>::S;
    constexpr int C = Shape<G>::C;
    const int64_t N = g.N;
    const double *pos = a.pos + DIM * off;
    const int8_t *mask = a.mask + off;
    const double *normal = a.normal ? a.normal + DIM * off : nullptr;
    double *row64 = a.row64 + S * off;
    float *row32 = a.row32 ? a.row32 + S * off : nullptr;
    double *ql64 = a.ql64 ? a.ql64 + S * off : nullptr;
    double *d64 = a.d64 ? a.d64 + (int64_t)NB * S * off : nullptr;
    double *qd64 = a.qd64 ? a.qd64 + (int64_t)NB * S * off : nullptr;
    double *rscale = a.rscale + off;
    int8_t *kind_out = a.kind + off;

    const int8_t mk = mask[k];
    int8_t kind;
    if (mk == 0) kind = KIND_VOID;
    else if (mk < 0) kind = KIND_INNER;
    else kind = (a.bc[(uint8_t)mk] == MCD_BC_NEUMANN) ? KIND_NEUMANN : KIND_DIRICHLET;

    auto write_identity = [&]() {
        for (int s = 0; s < S; ++s) {
            double v = (s == C) ? 1.0 : 0.0;
            row64[(int64_t)s * N + k] = v;
            if (row32) row32[(int64_t)s * N + k] = (float)v;
            if (ql64) ql64[(int64_t)s * N + k] = 0.0;
            if (d64)
                for (int c = 0; c < NB; ++c) d64[((int64_t)c * S + s) * N + k] = 0.0;
            if (qd64)
                for (int c = 0; c < NB; ++c) qd64[((int64_t)c * S + s) * N + k] = 0.0;
        }
        rscale[k] = 1.0;
    };

    kind_out[k] = kind;
    if (kind == KIND_VOID || kind == KIND_DIRICHLET) {
        write_identity();
        return;
    }

    int c[3] = {0, 0, 0};
    decode<DIM>(g, k, c);
    double xi[DIM];
    for (int d = 0; d < DIM; ++d) xi[d] = pos[(int64_t)d * N + k];
    const double inv_rs = 1.0 / r_s;
    const int nf = (kind == KIND_NEUMANN) ? DIM : NB;

    // ---- pass 1: moment matrix and sum_j w_j p_j over value neighbours ----
    double L[NB * (NB + 1) / 2];
    double acc[NB];
    for (int q = 0; q < NB * (NB + 1) / 2; ++q) L[q] = 0.0;
    for (int q = 0; q < NB; ++q) acc[q] = 0.0;
    // the 3x3 build keeps each neighbour's weight for pass 2 (registers:
    // the loops are unrolled), instead of evaluating the FP64 sqrt and exp a
    // second time; the wider stencils recompute it
    constexpr bool KEEP_W = (S == 9);
    double wkeep[KEEP_W ? S : 1];

#pragma unroll(KEEP_W ? S : 1)
    for (int s = 0; s < S; ++s) {
        if (s == C) continue;
        Nbr<DIM> nb = neighbour<G>(g, c, s);
        if (!nb.valid) continue;
        const int8_t mj = mask[nb.j];
        if (mj == 0) continue;
        const bool neu = (kind == KIND_INNER) && mj > 0 && a.bc[(uint8_t)mj] == MCD_BC_NEUMANN;
        double dx[DIM], X[DIM], r2 = 0.0;
        for (int d = 0; d < DIM; ++d) {
            dx[d] = (pos[(int64_t)d * N + nb.j] + nb.shift[d]) - xi[d];
            X[d] = dx[d] * inv_rs;
            r2 += dx[d] * dx[d];
        }
        const double w = mls_weight(sqrt(r2), a.weight_kind, r_e);
        if constexpr (KEEP_W) wkeep[s] = w;
        double p[NB];
        if (neu) {
            double n[DIM];
            for (int d = 0; d < DIM; ++d) n[d] = normal[(int64_t)d * N + nb.j];
            B::normal(X, n, p);
        } else {
            B::value(X, p);
            for (int q = 0; q < NB; ++q) acc[q] += w * p[q];
        }
        for (int r = 0; r < NB; ++r) {
            if (r >= nf) break;
            const double wp = w * p[r];
            for (int q = 0; q <= r; ++q) L[tri(r, q)] += wp * p[q];
        }
    }

    if (!cholesky<NB>(L, nf)) {
        atomicMin(a.bad, (unsigned long long)(off + k));
        write_identity();
        return;
    }

    // centre: -M^{-1} sum_j w_j p_j (from phi_j - phi_i)
    double cen[NB];
    for (int q = 0; q < NB; ++q) cen[q] = (q < nf) ? -acc[q] : 0.0;
    chol_solve<NB>(L, nf, cen);
    double scale[NB];
    for (int q = 0; q < NB; ++q)
        scale[q] = (B::order(q) == 1) ? inv_rs : inv_rs * inv_rs;
    for (int q = 0; q < NB; ++q) cen[q] *= scale[q];

    // Neumann DP: row = sigma n . grad, sigma = -1 / (r_s^2 n . grad_centre)
    double nrm[DIM];
    double sigma = 1.0;
    if (kind == KIND_NEUMANN) {
        double dcen = 0.0;
        for (int d = 0; d < DIM; ++d) {
            nrm[d] = normal[(int64_t)d * N + k];
            dcen += nrm[d] * cen[d];
        }
        if (!(dcen != 0.0) || !isfinite(dcen)) {
            atomicMin(a.bad, (unsigned long long)(off + k));
            write_identity();
            return;
        }
        sigma = -(inv_rs * inv_rs) / dcen;
    }
    rscale[k] = sigma;

    // ---- pass 2: per-slot weights ----
#pragma unroll(KEEP_W ? S : 1)
    for (int s = 0; s < S; ++s) {
        double z[NB];
        double zq[NB];
        for (int q = 0; q < NB; ++q) { z[q] = 0.0; zq[q] = 0.0; }
        if (s == C) {
            for (int q = 0; q < NB; ++q) z[q] = cen[q];
        } else {
            Nbr<DIM> nb = neighbour<G>(g, c, s);
            int8_t mj = nb.valid ? mask[nb.j] : (int8_t)0;
            if (mj != 0) {
                const bool neu = (kind == KIND_INNER) && mj > 0 && a.bc[(uint8_t)mj] == MCD_BC_NEUMANN;
                double dx[DIM], X[DIM], r2 = 0.0;
                for (int d = 0; d < DIM; ++d) {
                    dx[d] = (pos[(int64_t)d * N + nb.j] + nb.shift[d]) - xi[d];
                    X[d] = dx[d] * inv_rs;
                    r2 += dx[d] * dx[d];
                }
                double w;
                if constexpr (KEEP_W) w = wkeep[s];
                else w = mls_weight(sqrt(r2), a.weight_kind, r_e);
                double p[NB];
                if (neu) {
                    double n[DIM];
                    for (int d = 0; d < DIM; ++d) n[d] = normal[(int64_t)d * N + nb.j];
                    B::normal(X, n, p);
                    for (int q = 0; q < NB; ++q) zq[q] = (q < nf) ? w * p[q] * r_s : 0.0;
                    chol_solve<NB>(L, nf, zq);
                    for (int q = 0; q < NB; ++q) zq[q] *= scale[q];
                } else {
                    B::value(X, p);
                    for (int q = 0; q < NB; ++q) z[q] = (q < nf) ? w * p[q] : 0.0;
                    chol_solve<NB>(L, nf, z);
                    for (int q = 0; q < NB; ++q) z[q] *= scale[q];
                }
            }
        }
        double row = 0.0, ql = 0.0;
        if (kind == KIND_INNER) {
            for (int q = 0; q < NB; ++q)
                if (B::is_lap(q)) { row += z[q]; ql += zq[q]; }
        } else {
            for (int d = 0; d < DIM; ++d) row += nrm[d] * z[d];
            row *= sigma;
        }
        row64[(int64_t)s * N + k] = row;
        // FP32 rows are kept in difference form: the centre slot holds the
        // row sum, exactly 0 here (chi = 1 MLS reproduces constants), and the
        // SpMV forms sum_j c_ij (x_j - x_i); see spmv_kernel
        if (row32) row32[(int64_t)s * N + k] = (s == C) ? 0.0f : (float)row;
        if (ql64) ql64[(int64_t)s * N + k] = ql;
        if (d64)
            for (int q = 0; q < NB; ++q) d64[((int64_t)q * S + s) * N + k] = z[q];
        if (qd64)
            for (int q = 0; q < NB; ++q) qd64[((int64_t)q * S + s) * N + k] = zq[q];
    }
}


template <int G>
__global__ void __launch_bounds__(128) build_kernel(const __grid_constant__ BuildArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.g.N) return;
    build_dp<G>(a, a.g, 0, k, a.r_e, a.r_s);
}

// Batched build: the blocks of system i start at blk_start[i]; geo[i] and
// off[i] give its geometry and DP offset; r_e and r_s are multiples of its l0.
template <int G>
__global__ void __launch_bounds__(128) build_batch_kernel(const __grid_constant__ BuildArgs a,
                                                          const Geo *__restrict__ geo,
                                                          const int64_t *__restrict__ off,
                                                          const int *__restrict__ blk_start, int nsys) {
    int lo = 0, hi = nsys - 1;
    const int blk = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_start[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    const Geo g = geo[lo];
    const int64_t k = (int64_t)(blk - blk_start[lo]) * blockDim.x + threadIdx.x;
    if (k >= g.N) return;
    build_dp<G>(a, g, off[lo], k, a.r_e * g.l0, a.r_s * g.l0);
}

cudaError_t launch_build_batch(const BatchBuildDesc &d, cudaStream_t stream) {
    BuildArgs a;
    memset(&a, 0, sizeof(a));
    a.pos = d.pos;
    a.mask = d.mask;
    a.normal = nullptr;
    for (int b = 0; b < 128; ++b) a.bc[b] = d.prm->bc_kind[b];
    a.weight_kind = d.prm->weight_kind;
    a.r_e = d.prm->r_e;
    a.r_s = d.prm->r_s;
    a.row64 = d.row64;
    a.row32 = d.row32;
    a.rscale = d.rscale;
    a.kind = d.kind;
    a.bad = d.bad;
    MCD_KLAUNCH(MCD_K_BUILD, stream, build_batch_kernel<2><<<d.nblocks, 128, 0, stream>>>(
        a, d.geo, d.off, d.blk_start, d.nsys));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// y = A x with the PPE rows: the matrix-free stencil SpMV.
// FP64 rows are in matrix form, y_i = sum_s c_is x_js.  FP32 rows are in
// difference form, y_i = c_iC x_i + sum_{s != C} c_is (x_js - x_i) with the
// centre slot holding the row sum: for a smooth x the products then carry
// O(l0) differences instead of O(1) values, which keeps the cancellation of
// the O(1/l0^2) weights from consuming the FP32 mantissa; the products are
// split exactly with fma and summed with TwoSum (double-float accumulation).
// ---------------------------------------------------------------------------
template <typename T, int G>
__global__ void __launch_bounds__(256) spmv_kernel(Geo g, const T *__restrict__ row,
                                                   const T *__restrict__ x, T *__restrict__ y) {
    constexpr int DIM = Shape<G>::dim;
    constexpr int S = Shape<G>::S;
    constexpr int C = Shape<G>::C;
    constexpr bool diff_form = sizeof(T) == 4;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int c[3] = {0, 0, 0};
    decode<DIM>(g, k, c);
    const T xi = x[k];
    if (diff_form) {
        // compensated: exact products (fma) summed by TwoSum into (hi, lo)
        float hi = (float)row[(int64_t)C * N + k] * (float)xi, lo = 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (s == C) continue;
            Nbr<DIM> nb = neighbour<G>(g, c, s);
            const float w = (float)row[(int64_t)s * N + k];
            // _rn intrinsics: never contracted into fused multiply-adds
            const float d = __fsub_rn((float)x[nb.j], (float)xi);
            const float p = __fmul_rn(w, d);
            const float pe = __fmaf_rn(w, d, -p);
            const float sum = __fadd_rn(hi, p);
            const float bb = __fsub_rn(sum, hi);
            lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(p, bb)), pe));
            hi = sum;
        }
        y[k] = (T)__fadd_rn(hi, lo);
        return;
    }
    T acc = (T)0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        Nbr<DIM> nb = neighbour<G>(g, c, s);
        acc += row[(int64_t)s * N + k] * x[nb.j];
    }
    y[k] = acc;
}

// The 2D 3x3 SpMV, tiled for HBM: one block of 256 threads per tile of
// (32 VEC) x 8 cells; thread (tx, ty) owns the VEC consecutive cells
// (i0 + VEC tx + v, j0 + ty), v < VEC.  x of the tile and its one-cell halo
// is staged in shared memory (wrapped on periodic axes, clamped otherwise,
// which is how neighbour() maps a missing neighbour: onto the cell itself),
// each slot's weights of the VEC cells arrive in one 16-byte streaming load,
// and y leaves in one 16-byte store.  Per cell the products and the order of
// their sum are those of spmv_kernel.  VEC > 1 needs n0 % VEC == 0.
__device__ __forceinline__ int halo_coord(int v, int n, int per) {
    if (v < 0) return per ? v + n : 0;
    if (v >= n) return per ? v - n : n - 1;
    return v;
}

template <typename T, int VEC>
__global__ void __launch_bounds__(256) spmv2d_tiled(Geo g, const T *__restrict__ row,
                                                    const T *__restrict__ x, T *__restrict__ y) {
    constexpr int TX = 32 * VEC, TY = 8;
    constexpr int OFF = 16 / sizeof(T);    // shared column of cell i0: 16-byte aligned
    constexpr int XS = TX + 2 * OFF;
    constexpr int C = 4;
    constexpr bool diff_form = sizeof(T) == 4;
    __shared__ __align__(16) T xs[TY + 2][XS];
    const int n0 = g.n[0], n1 = g.n[1];
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i = i0 + VEC * tx, j = j0 + ty;
    const bool in = i < n0 && j < n1;
    const int64_t N = g.N;
    const int64_t k = (int64_t)i + (int64_t)n0 * j;
    // the weights first: their loads are in flight while x is staged
    T w[9][VEC];
#pragma unroll
    for (int sl = 0; sl < 9; ++sl) {
        const T *src = row + (int64_t)sl * N + k;
        if (!in) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) w[sl][v] = (T)0;
        } else if constexpr (VEC == 4) {
            const float4 v4 = __ldcs(reinterpret_cast<const float4 *>(src));
            w[sl][0] = v4.x; w[sl][1] = v4.y; w[sl][2] = v4.z; w[sl][3] = v4.w;
        } else if constexpr (VEC == 2) {
            const double2 v2 = __ldcs(reinterpret_cast<const double2 *>(src));
            w[sl][0] = v2.x; w[sl][1] = v2.y;
        } else {
            w[sl][0] = __ldcs(src);
        }
    }
    for (int h = threadIdx.x; h < (TY + 2) * (TX + 2); h += 256) {
        const int hy = h / (TX + 2), hx = h - hy * (TX + 2);
        // columns and rows past the mesh's own halo (ragged tiles) are
        // clamped into it: they are loaded but never used
        const int gx = halo_coord(min(i0 + hx - 1, n0), n0, g.per[0]);
        const int gy = halo_coord(min(j0 + hy - 1, n1), n1, g.per[1]);
        xs[hy][OFF - 1 + hx] = __ldg(x + (int64_t)gx + (int64_t)n0 * gy);
    }
    __syncthreads();
    if (!in) return;
    T xr[3][VEC + 2];
#pragma unroll
    for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int c = 0; c < VEC + 2; ++c) xr[dj][c] = xs[ty + dj][OFF - 1 + VEC * tx + c];
    T out[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const T xi = xr[1][v + 1];
        if constexpr (diff_form) {
            float hi = (float)w[C][v] * (float)xi, lo = 0.0f;
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) {
                if (sl == C) continue;
                const float wv = (float)w[sl][v];
                const float d = __fsub_rn((float)xr[sl / 3][v + 1 + sl % 3 - 1], (float)xi);
                const float pr = __fmul_rn(wv, d);
                const float pe = __fmaf_rn(wv, d, -pr);
                const float sum = __fadd_rn(hi, pr);
                const float bb = __fsub_rn(sum, hi);
                lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(pr, bb)), pe));
                hi = sum;
            }
            out[v] = (T)__fadd_rn(hi, lo);
        } else {
            T acc = (T)0;
#pragma unroll
            for (int sl = 0; sl < 9; ++sl) acc = fma(w[sl][v], xr[sl / 3][v + 1 + sl % 3 - 1], acc);
            out[v] = acc;
        }
    }
    if constexpr (VEC == 4) {
        __stcs(reinterpret_cast<float4 *>(y + k), make_float4(out[0], out[1], out[2], out[3]));
    } else if constexpr (VEC == 2) {
        __stcs(reinterpret_cast<double2 *>(y + k), make_double2(out[0], out[1]));
    } else {
        y[k] = out[0];
    }
}

// The 2D 3x3 SpMV streamed by TMA (non-periodic meshes): a persistent
// launch, two blocks per SM, whose blocks take tiles of TX x 8 cells in turn
// (tile blockIdx.x + k gridDim.x).  Thread 0 keeps NS stages in flight; a
// stage is two cp.async.bulk.tensor copies completing on its mbarrier: the
// tile's nine weight slots (box TX x 8 x 9 of the rows as a [9][n1][n0]
// tensor) and x over the tile and its halo (box (TX + 2 HP) x 10 of x as a
// [n1][n0] tensor, from column i0 - HP so that the copy starts on a 16-byte
// boundary).  Copies reaching past the mesh fill zeros; a missing neighbour
// carries zero weight (the build leaves it out of the fit), so it adds
// nothing, as in spmv_kernel.  Per cell the arithmetic and its order are
// spmv_kernel's.  Every wait is bounded: on a timeout the block raises *err,
// stops issuing, waits (bounded) for the copies it has in flight and returns.
template <typename T> struct SpmvTma {
    static constexpr int VEC = 16 / (int)sizeof(T);   // cells per thread: 4 (FP32), 2 (FP64)
    static constexpr int TX = 32 * VEC, TY = 8;
    static constexpr int HP = VEC;                      // x columns loaded on each side
    static constexpr int XW = TX + 2 * HP;              // x box width (544 bytes)
    static constexpr unsigned ROWS_BYTES = 9u * TY * TX * sizeof(T);
    static constexpr unsigned X_BYTES = (TY + 2u) * XW * sizeof(T);
    static constexpr unsigned X_PAD = (X_BYTES + 127u) / 128u * 128u;
    static constexpr unsigned STAGE = ROWS_BYTES + X_PAD;   // 128-byte aligned stages
    static constexpr int NS = 2;
    static constexpr size_t SMEM = (size_t)NS * STAGE;
};

__device__ __forceinline__ uint32_t spmv_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool spmv_wait(uint64_t *mbar, uint32_t parity, long long limit) {
    const uint32_t mb = spmv_smem(mbar);
    uint32_t done = 0;
    for (long long polls = 0; !done; ++polls) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
        if (!done && polls >= limit) return false;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256, 2) spmv2d_tma(const __grid_constant__ CUtensorMap rows_map,
                                                     const __grid_constant__ CUtensorMap x_map, int n0, int n1,
                                                     int tiles_x, int ntiles, T *__restrict__ y, int *err,
                                                     long long spin_limit) {
    using P = SpmvTma<T>;
    constexpr int VEC = P::VEC, TX = P::TX, TY = P::TY, XW = P::XW, C = 4;
    constexpr bool diff_form = sizeof(T) == 4;
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[P::NS];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const int mine = (blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        for (int b = 0; b < P::NS; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(spmv_smem(mbar + b)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    auto issue = [&](int k) {   // thread 0: tile k of this block into stage k % NS
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        unsigned char *st = smem + (size_t)(k % P::NS) * P::STAGE;
        const uint32_t mb = spmv_smem(mbar + k % P::NS);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                     "r"(P::ROWS_BYTES + P::X_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(spmv_smem(st)),
            "l"(reinterpret_cast<uint64_t>(&rows_map)), "r"(x0), "r"(y0), "r"(0), "r"(mb)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(spmv_smem(st + P::ROWS_BYTES)),
            "l"(reinterpret_cast<uint64_t>(&x_map)), "r"(x0 - P::HP), "r"(y0 - 1), "r"(mb)
            : "memory");
    };
    if (tid == 0)
        for (int k = 0; k < P::NS && k < mine; ++k) issue(k);
    const int tx = tid & 31, ty = tid >> 5;
    int k = 0;
    for (; k < mine; ++k) {
        const int b = k % P::NS;
        const bool ok = spmv_wait(mbar + b, (uint32_t)((k / P::NS) & 1), spin_limit);
        if (__syncthreads_or(!ok)) break;
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        const int i = (t % tiles_x) * TX + VEC * tx, j = (t / tiles_x) * TY + ty;
        const T *W = reinterpret_cast<const T *>(smem + (size_t)b * P::STAGE);
        const T *X = reinterpret_cast<const T *>(smem + (size_t)b * P::STAGE + P::ROWS_BYTES);
        T w[9][VEC];
#pragma unroll
        for (int sl = 0; sl < 9; ++sl) {
            const V wv = *reinterpret_cast<const V *>(W + (sl * TY + ty) * TX + VEC * tx);
            if constexpr (VEC == 4) {
                w[sl][0] = wv.x; w[sl][1] = wv.y; w[sl][2] = wv.z; w[sl][3] = wv.w;
            } else {
                w[sl][0] = wv.x; w[sl][1] = wv.y;
            }
        }
        // x of cells i - 1 .. i + VEC of rows j - 1 .. j + 1: three aligned
        // vectors per row (the thread's own and its two neighbours')
        T xr[3][VEC + 2];
#pragma unroll
        for (int dj = 0; dj < 3; ++dj) {
            const T *row = X + (ty + dj) * XW;
            const V lo = *reinterpret_cast<const V *>(row + VEC * tx);
            const V mid = *reinterpret_cast<const V *>(row + VEC * (tx + 1));
            const V hi = *reinterpret_cast<const V *>(row + VEC * (tx + 2));
            if constexpr (VEC == 4) {
                xr[dj][0] = lo.w; xr[dj][1] = mid.x; xr[dj][2] = mid.y; xr[dj][3] = mid.z; xr[dj][4] = mid.w;
                xr[dj][5] = hi.x;
            } else {
                xr[dj][0] = lo.y; xr[dj][1] = mid.x; xr[dj][2] = mid.y; xr[dj][3] = hi.x;
            }
        }
        __syncthreads();   // every thread has its operands: stage b may be refilled
        if (tid == 0 && k + P::NS < mine) issue(k + P::NS);
        if (i >= n0 || j >= n1) continue;
        T out[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const T xi = xr[1][v + 1];
            if constexpr (diff_form) {
                float hi = (float)w[C][v] * (float)xi, lo = 0.0f;
#pragma unroll
                for (int sl = 0; sl < 9; ++sl) {
                    if (sl == C) continue;
                    const float wv = (float)w[sl][v];
                    const float d = __fsub_rn((float)xr[sl / 3][v + 1 + sl % 3 - 1], (float)xi);
                    const float pr = __fmul_rn(wv, d);
                    const float pe = __fmaf_rn(wv, d, -pr);
                    const float sum = __fadd_rn(hi, pr);
                    const float bb = __fsub_rn(sum, hi);
                    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(pr, bb)), pe));
                    hi = sum;
                }
                out[v] = (T)__fadd_rn(hi, lo);
            } else {
                T acc = (T)0;
#pragma unroll
                for (int sl = 0; sl < 9; ++sl) acc = fma(w[sl][v], xr[sl / 3][v + 1 + sl % 3 - 1], acc);
                out[v] = acc;
            }
        }
        const int64_t kk = (int64_t)i + (int64_t)n0 * j;
        if constexpr (VEC == 4) {
            __stcs(reinterpret_cast<float4 *>(y + kk), make_float4(out[0], out[1], out[2], out[3]));
        } else {
            __stcs(reinterpret_cast<double2 *>(y + kk), make_double2(out[0], out[1]));
        }
    }
    if (k < mine && tid == 0) {
        // a wait gave up: report it and let the copies in flight land
        // (bounded) before the block's shared memory is released
        atomicExch(err, 1);
        for (int q = k; q < mine && q < k + P::NS; ++q)
            if (!spmv_wait(mbar + q % P::NS, (uint32_t)((q / P::NS) & 1), spin_limit)) break;
    }
}

typedef CUresult (*SpmvEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static SpmvEncodeFn spmv_encoder() {
    static SpmvEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<SpmvEncodeFn>(ptr);
    }
    return fn;
}

// Launch spmv2d_tma if the layout allows it (non-periodic 2D 3x3, n0 a
// multiple of the vector width, 16-byte aligned arrays); false otherwise.
template <typename T>
static bool launch_spmv_tma(const mcd_stencils *st, const T *row, const T *x, T *y, cudaStream_t stream) {
    using P = SpmvTma<T>;
    const Geo &g = st->geo;
    if (st->shape != 2 || g.per[0] || g.per[1] || g.n[0] % P::VEC != 0) return false;
    if ((uintptr_t)row % 16 || (uintptr_t)x % 16 || (uintptr_t)y % 16) return false;
    if (((uint64_t)g.N * sizeof(T)) % 16) return false;   // slot stride of the rows
    SpmvEncodeFn enc = spmv_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t n0 = (cuuint64_t)g.n[0], n1 = (cuuint64_t)g.n[1], es = sizeof(T);
    CUtensorMap rows_map, x_map;
    const cuuint64_t rdims[3] = {n0, n1, 9};
    const cuuint64_t rstr[2] = {n0 * es, n0 * n1 * es};
    const cuuint32_t rbox[3] = {(cuuint32_t)P::TX, (cuuint32_t)P::TY, 9};
    const cuuint32_t ones[3] = {1, 1, 1};
    if (enc(&rows_map, dt, 3, const_cast<T *>(row), rdims, rstr, rbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t xdims[2] = {n0, n1};
    const cuuint64_t xstr[1] = {n0 * es};
    const cuuint32_t xbox[2] = {(cuuint32_t)P::XW, (cuuint32_t)(P::TY + 2)};
    if (enc(&x_map, dt, 2, const_cast<T *>(x), xdims, xstr, xbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    static int sms[64] = {0};
    static bool attr_set[2][64] = {{false}};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    if (!attr_set[sizeof(T) == 8][dev]) {
        if (cudaFuncSetAttribute(spmv2d_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM) !=
            cudaSuccess)
            return false;
        attr_set[sizeof(T) == 8][dev] = true;
    }
    const int tiles_x = (g.n[0] + P::TX - 1) / P::TX, tiles_y = (g.n[1] + P::TY - 1) / P::TY;
    const int ntiles = tiles_x * tiles_y;
    const int grid = std::min(ntiles, 2 * sms[dev]);
    {
        KTimer kt(MCD_K_OTHER, stream);
        spmv2d_tma<T><<<grid, 256, P::SMEM, stream>>>(rows_map, x_map, g.n[0], g.n[1], tiles_x, ntiles, y,
                                                      st->spmv_err, 1ll << 22);
    }
    return true;
}

// b: inner DP f - sum QL * bnd (Neumann neighbours); boundary DP rscale * bnd.
template <int G>
__global__ void rhs_kernel(Geo g, const int8_t *__restrict__ kind, const double *__restrict__ ql,
                           const double *__restrict__ rscale, const double *__restrict__ rhs,
                           const double *__restrict__ bnd, double *__restrict__ b) {
    constexpr int DIM = Shape<G>::dim;
    constexpr int S = Shape<G>::S;
    const int64_t N = g.N;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int8_t kd = kind[k];
    double out = 0.0;
    if (kd == KIND_INNER) {
        out = rhs[k];
        if (ql) {
            int c[3] = {0, 0, 0};
            decode<DIM>(g, k, c);
            for (int s = 0; s < S; ++s) {
                const double q = ql[(int64_t)s * N + k];
                if (q != 0.0) {
                    Nbr<DIM> nb = neighbour<G>(g, c, s);
                    out -= q * bnd[nb.j];
                }
            }
        }
    } else if (kd == KIND_DIRICHLET || kd == KIND_NEUMANN) {
        out = rscale[k] * bnd[k];
    }
    b[k] = out;
}

template <typename T>
static cudaError_t dmalloc(T **p, size_t count) {
    return cudaMalloc((void **)p, count * sizeof(T));
}

void free_workspace(mcd_stencils *st);

static void free_arrays(mcd_stencils *st) {
    cudaFree(st->row64);
    cudaFree(st->row32);
    cudaFree(st->ql64);
    cudaFree(st->d64);
    cudaFree(st->qd64);
    cudaFree(st->rscale);
    cudaFree(st->kind);
    cudaFree(st->off16);
    cudaFree(st->bad_dp);
    cudaFree(st->spmv_err);
}

static bool same_layout(const mcd_stencils *st, const mcd_mesh &m, const mcd_mls_params &p) {
    if (st->mesh.dim != m.dim) return false;
    for (int d = 0; d < 3; ++d)
        if (st->mesh.n[d] != m.n[d]) return false;
    int has_neu = 0;
    for (int b = 1; b < 128; ++b) has_neu |= (p.bc_kind[b] == MCD_BC_NEUMANN);
    return st->prm.precision == p.precision && st->prm.want_derivs == p.want_derivs &&
           st->has_neumann == has_neu && st->support == (p.support == 0 ? 1 : p.support);
}

}  // namespace mcd

using namespace mcd;

static mcd_status validate_mesh(const mcd_mesh *m) {
    MCD_CHECK_ARG(m != nullptr, "mesh is NULL");
    MCD_CHECK_ARG(m->dim == 2 || m->dim == 3, "mesh.dim must be 2 or 3");
    for (int d = 0; d < m->dim; ++d) MCD_CHECK_ARG(m->n[d] >= 3, "mesh.n[d] must be >= 3");
    if (m->dim == 2) MCD_CHECK_ARG(m->n[2] == 1, "2D mesh needs n[2] = 1");
    MCD_CHECK_ARG(m->l0 > 0.0, "mesh.l0 must be positive");
    return MCD_OK;
}

extern "C" mcd_status mcd_build_stencils(const mcd_mesh *mesh, const double *pos_dev,
                                         const int8_t *mask_dev, const double *normal_dev,
                                         const mcd_mls_params *prm, mcd_stencils **st,
                                         mcd_stream_t stream) {
    mcd_status v = validate_mesh(mesh);
    if (v != MCD_OK) return v;
    MCD_CHECK_ARG(pos_dev && mask_dev && prm && st, "NULL argument");
    MCD_CHECK_ARG(prm->r_e > 0.0 && prm->r_s > 0.0, "r_e and r_s must be positive");
    MCD_CHECK_ARG(prm->weight_kind == MCD_W_GAUSS || prm->weight_kind == MCD_W_COS2 ||
                      prm->weight_kind == MCD_W_LSMPS,
                  "unknown weight_kind");
    const int support = prm->support == 0 ? 1 : prm->support;
    const int shape = shape_code(mesh->dim, support);
    MCD_CHECK_ARG(shape != 0, "support must be 1 (3x3, 3x3x3) or 4 (2D 9x9)");
    for (int d = 0; d < mesh->dim; ++d)
        MCD_CHECK_ARG(!mesh->periodic[d] || mesh->n[d] >= 2 * support + 1,
                      "a periodic axis needs at least 2 support + 1 cells");
    MCD_CHECK_ARG(prm->precision == MCD_FP64 || prm->precision == MCD_MIXED, "unknown precision");
    int has_neu = 0;
    for (int b = 1; b < 128; ++b) has_neu |= (prm->bc_kind[b] == MCD_BC_NEUMANN);
    MCD_CHECK_ARG(!has_neu || normal_dev, "normals are required when a boundary id is Neumann");

    mcd_stencils *h = *st;
    if (h && !same_layout(h, *mesh, *prm)) {
        set_error("existing stencil handle has a different mesh size or options");
        return MCD_EINVAL;
    }
    const Geo g = make_geo(*mesh);
    const int S = (mesh->dim == 2) ? (2 * support + 1) * (2 * support + 1)
                                   : (2 * support + 1) * (2 * support + 1) * (2 * support + 1);
    const int nb = (mesh->dim == 2) ? 5 : 9;
    const int64_t N = g.N;
    if (!h) {
        h = new mcd_stencils();
        h->mesh = *mesh;
        h->prm = *prm;
        h->geo = g;
        h->S = S;
        h->support = support;
        h->shape = shape;
        h->nb = nb;
        h->has_neumann = has_neu;
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        chk(dmalloc(&h->row64, (size_t)S * N));
        if (prm->precision == MCD_MIXED) chk(dmalloc(&h->row32, (size_t)S * N));
        if (has_neu) chk(dmalloc(&h->ql64, (size_t)S * N));
        if (prm->want_derivs) {
            chk(dmalloc(&h->d64, (size_t)nb * S * N));
            if (has_neu) chk(dmalloc(&h->qd64, (size_t)nb * S * N));
        }
        chk(dmalloc(&h->rscale, (size_t)N));
        chk(dmalloc(&h->kind, (size_t)N));
        if (mesh->dim == 2) chk(dmalloc(&h->off16, (size_t)2 * N));
        chk(dmalloc(&h->bad_dp, 1));
        chk(dmalloc(&h->spmv_err, 1));
        if (e == cudaSuccess) chk(cudaMemset(h->spmv_err, 0, sizeof(int)));
        if (e != cudaSuccess) {
            free_arrays(h);
            delete h;
            set_error(std::string("stencil allocation: ") + cudaGetErrorString(e));
            return MCD_ENOMEM;
        }
        *st = h;
    }
    h->mesh = *mesh;
    h->geo = g;
    h->prm = *prm;
    h->has_neumann = has_neu;

    MCD_CUDA_TRY(cudaMemsetAsync(h->bad_dp, 0xff, sizeof(unsigned long long), stream));
    BuildArgs a;
    a.g = g;
    a.pos = pos_dev;
    a.mask = mask_dev;
    a.normal = normal_dev;
    for (int b = 0; b < 128; ++b) a.bc[b] = prm->bc_kind[b];
    a.weight_kind = prm->weight_kind;
    a.r_e = prm->r_e;
    a.r_s = prm->r_s;
    a.row64 = h->row64;
    a.row32 = h->row32;
    a.ql64 = h->ql64;
    a.d64 = h->d64;
    a.qd64 = h->qd64;
    a.rscale = h->rscale;
    a.kind = h->kind;
    a.bad = h->bad_dp;
    const int threads = 128;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    if (shape == 2)
        MCD_KLAUNCH(MCD_K_BUILD, stream, build_kernel<2><<<blocks, threads, 0, stream>>>(a));
    else if (shape == 3)
        MCD_KLAUNCH(MCD_K_BUILD, stream, build_kernel<3><<<blocks, threads, 0, stream>>>(a));
    else
        MCD_KLAUNCH(MCD_K_BUILD, stream, build_kernel<9><<<blocks, threads, 0, stream>>>(a));
    MCD_LAUNCH_CHECK();
    MCD_CUDA_TRY(cnn_store_offsets(h, pos_dev, mask_dev, stream));
    return MCD_OK;
}

extern "C" mcd_status mcd_stencils_check(const mcd_stencils *st, int64_t *first_bad_dp,
                                         mcd_stream_t stream) {
    MCD_CHECK_ARG(st, "NULL handle");
    unsigned long long bad = 0;
    int spmv_err = 0;
    MCD_CUDA_TRY(cudaMemcpyAsync(&bad, st->bad_dp, sizeof(bad), cudaMemcpyDeviceToHost, stream));
    MCD_CUDA_TRY(cudaMemcpyAsync(&spmv_err, st->spmv_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    MCD_CUDA_TRY(cudaStreamSynchronize(stream));
    if (spmv_err) {
        set_error("a TMA-streamed SpMV of this handle gave up waiting for its copies (bounded wait)");
        return MCD_ETIMEOUT;
    }
    const bool fail = bad != ~0ull;
    if (first_bad_dp) *first_bad_dp = fail ? (int64_t)bad : -1;
    if (fail) {
        set_error("singular MLS moment matrix at DP " + std::to_string(bad));
        return MCD_ESINGULAR;
    }
    return MCD_OK;
}

extern "C" void mcd_stencils_destroy(mcd_stencils *st) {
    if (!st) return;
    free_workspace(st);
    free_arrays(st);
    delete st;
}

extern "C" mcd_status mcd_stencils_array(const mcd_stencils *st, int which,
                                         const void **dev_ptr, int64_t *count) {
    MCD_CHECK_ARG(st && dev_ptr, "NULL argument");
    const int64_t N = st->geo.N;
    const void *p = nullptr;
    int64_t n = 0;
    switch (which) {
        case MCD_ARR_ROW64: p = st->row64; n = (int64_t)st->S * N; break;
        case MCD_ARR_ROW32: p = st->row32; n = st->row32 ? (int64_t)st->S * N : 0; break;
        case MCD_ARR_QL64: p = st->ql64; n = st->ql64 ? (int64_t)st->S * N : 0; break;
        case MCD_ARR_D64: p = st->d64; n = st->d64 ? (int64_t)st->nb * st->S * N : 0; break;
        case MCD_ARR_QD64: p = st->qd64; n = st->qd64 ? (int64_t)st->nb * st->S * N : 0; break;
        case MCD_ARR_RSCALE: p = st->rscale; n = N; break;
        case MCD_ARR_KIND: p = st->kind; n = N; break;
        default: set_error("unknown array id"); return MCD_EINVAL;
    }
    *dev_ptr = p;
    if (count) *count = n;
    return MCD_OK;
}

extern "C" mcd_status mcd_stencils_copy(const mcd_stencils *st, int which, void *dst_dev,
                                        mcd_stream_t stream) {
    MCD_CHECK_ARG(dst_dev, "NULL destination");
    const void *src = nullptr;
    int64_t count = 0;
    mcd_status s = mcd_stencils_array(st, which, &src, &count);
    if (s != MCD_OK) return s;
    MCD_CHECK_ARG(src && count > 0, "array not kept by this handle");
    size_t elem = 8;
    if (which == MCD_ARR_ROW32) elem = 4;
    if (which == MCD_ARR_KIND) elem = 1;
    MCD_CUDA_TRY(cudaMemcpyAsync(dst_dev, src, (size_t)count * elem, cudaMemcpyDeviceToDevice, stream));
    return MCD_OK;
}

extern "C" mcd_status mcd_apply_laplacian(const mcd_stencils *st, const void *x_dev,
                                          void *y_dev, int dtype, mcd_stream_t stream) {
    MCD_CHECK_ARG(st && x_dev && y_dev, "NULL argument");
    MCD_CHECK_ARG(x_dev != y_dev, "x and y must not alias");
    const int64_t N = st->geo.N;
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    const int n0 = st->geo.n[0], n1 = st->geo.n[1];
    const bool tiled = st->shape == 2 && (n1 + 7) / 8 <= 65535;
    // the vector paths load 16-byte groups of the rows and store y the same
    // way: the rows and y must start on 16-byte boundaries (a system of a
    // batch starts at an arbitrary DP offset inside the batch's arrays)
    auto al16 = [](const void *q) { return ((uintptr_t)q % 16) == 0; };
    if (dtype == MCD_DT_F64) {
        const double *row = st->row64;
        const double *x = (const double *)x_dev;
        double *y = (double *)y_dev;
        // FP64: the shared-memory tiles (the product is bound by the FP64
        // pipe, 9 DFMA per DP, which TMA staging does not relieve: 0.278 ms
        // against 0.312 ms at 4096^2)
        if (tiled && n0 % 2 == 0 && al16(row) && al16(y))
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv2d_tiled<double, 2><<<dim3((n0 + 63) / 64, (n1 + 7) / 8), threads, 0, stream>>>(st->geo, row, x, y));
        else if (tiled)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv2d_tiled<double, 1><<<dim3((n0 + 31) / 32, (n1 + 7) / 8), threads, 0, stream>>>(st->geo, row, x, y));
        else if (st->shape == 2)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<double, 2><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
        else if (st->shape == 3)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<double, 3><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
        else
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<double, 9><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
    } else if (dtype == MCD_DT_F32) {
        MCD_CHECK_ARG(st->row32, "FP32 rows need an MCD_MIXED stencil handle");
        const float *row = st->row32;
        const float *x = (const float *)x_dev;
        float *y = (float *)y_dev;
        if (launch_spmv_tma<float>(st, row, x, y, stream))
            ;
        else if (tiled && n0 % 4 == 0 && al16(row) && al16(y))
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv2d_tiled<float, 4><<<dim3((n0 + 127) / 128, (n1 + 7) / 8), threads, 0, stream>>>(st->geo, row, x, y));
        else if (tiled)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv2d_tiled<float, 1><<<dim3((n0 + 31) / 32, (n1 + 7) / 8), threads, 0, stream>>>(st->geo, row, x, y));
        else if (st->shape == 2)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<float, 2><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
        else if (st->shape == 3)
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<float, 3><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
        else
            MCD_KLAUNCH(MCD_K_OTHER, stream, spmv_kernel<float, 9><<<blocks, threads, 0, stream>>>(st->geo, row, x, y));
    } else {
        set_error("unknown dtype");
        return MCD_EINVAL;
    }
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

extern "C" mcd_status mcd_assemble_rhs(const mcd_stencils *st, const double *rhs_dev,
                                       const double *bnd_dev, double *b_dev, mcd_stream_t stream) {
    MCD_CHECK_ARG(st && rhs_dev && bnd_dev && b_dev, "NULL argument");
    const int64_t N = st->geo.N;
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    const double *ql = st->has_neumann ? st->ql64 : nullptr;
    if (st->shape == 2)
        MCD_KLAUNCH(MCD_K_OTHER, stream, rhs_kernel<2><<<blocks, threads, 0, stream>>>(st->geo, st->kind, ql, st->rscale, rhs_dev, bnd_dev, b_dev));
    else if (st->shape == 3)
        MCD_KLAUNCH(MCD_K_OTHER, stream, rhs_kernel<3><<<blocks, threads, 0, stream>>>(st->geo, st->kind, ql, st->rscale, rhs_dev, bnd_dev, b_dev));
    else
        MCD_KLAUNCH(MCD_K_OTHER, stream, rhs_kernel<9><<<blocks, threads, 0, stream>>>(st->geo, st->kind, ql, st->rscale, rhs_dev, bnd_dev, b_dev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

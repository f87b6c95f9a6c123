// Internal helpers shared by the translation units of libmcd (not part of
// the C ABI).  Error plumbing, the stencil handle layout, the slot
// geometry of the 3x3 / 3x3x3 compact support and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mcd.h"

namespace mcd {

void set_error(const std::string &msg);

#define MCD_CUDA_TRY(call)                                                    \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            ::mcd::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return MCD_ECUDA;                                                 \
        }                                                                     \
    } while (0)

#define MCD_CHECK_ARG(cond, msg)                                              \
    do {                                                                      \
        if (!(cond)) {                                                        \
            ::mcd::set_error(msg);                                            \
            return MCD_EINVAL;                                                \
        }                                                                     \
    } while (0)

#define MCD_LAUNCH_CHECK()                                                    \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) {                                              \
            ::mcd::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_)); \
            return MCD_ECUDA;                                                 \
        }                                                                     \
    } while (0)

// Slot s of the compact support: 2D s = (di+1) + 3 (dj+1); 3D adds 9 (dl+1).
// Kind codes written per DP.
enum : int8_t { KIND_VOID = 0, KIND_INNER = 1, KIND_DIRICHLET = 2, KIND_NEUMANN = 3 };

// Geometry passed by value to kernels.
struct Geo {
    int dim;
    int n[3];
    int per[3];
    double l0;
    double org[3];
    double len[3];   // n[d] * l0 (periodic shift)
    int64_t N;
};

// Stencil shape of a solve: the (2R+1)^dim background cells around a DP's
// own cell.  G = 2: 2D 3x3, G = 3: 3D 3x3x3 (the MCD stencils of Sec. 3.2),
// G = 9: 2D 9x9 (the expanded stencil of Sec. 4.1).  Slot s holds the cell
// at offset (s % W - R, (s / W) % W - R, s / W^2 - R), W = 2R + 1.
template <int D, int RR> struct ShapeOf {
    static constexpr int dim = D;
    static constexpr int R = RR;
    static constexpr int W = 2 * RR + 1;
    static constexpr int S = (D == 2) ? W * W : W * W * W;
    static constexpr int C = S / 2;
};
template <int G> struct Shape;
template <> struct Shape<2> : ShapeOf<2, 1> {};
template <> struct Shape<3> : ShapeOf<3, 1> {};
template <> struct Shape<9> : ShapeOf<2, 4> {};

template <int G>
__host__ __device__ __forceinline__ void slot_offset(int s, int *o) {
    using SH = Shape<G>;
    o[0] = s % SH::W - SH::R;
    o[1] = (s / SH::W) % SH::W - SH::R;
    o[2] = (SH::dim == 3) ? s / (SH::W * SH::W) - SH::R : 0;
}

// Shape code of a (dim, support radius) pair; 0 if unsupported.
inline int shape_code(int dim, int support) {
    if (support == 1) return dim;
    if (support == 4 && dim == 2) return 9;
    return 0;
}

inline Geo make_geo(const mcd_mesh &m) {
    Geo g;
    g.dim = m.dim;
    g.N = 1;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = (d < m.dim) ? m.n[d] : 1;
        g.per[d] = (d < m.dim) ? (m.periodic[d] ? 1 : 0) : 0;
        g.org[d] = (d < m.dim) ? m.origin[d] : 0.0;
        g.len[d] = g.n[d] * m.l0;
        g.N *= g.n[d];
    }
    g.l0 = m.l0;
    return g;
}

// Neighbour of cell coordinate c along one axis with offset o: returns the
// wrapped / validated coordinate and the position shift a periodic wrap
// implies (x_j + shift is the minimum image seen from the centre cell).
__device__ __forceinline__ int nb_coord(int c, int o, int n, int per, double len,
                                        double &shift, bool &valid) {
    int v = c + o;
    shift = 0.0;
    if (v < 0) {
        if (per) { v += n; shift = -len; } else { valid = false; v = c; }
    } else if (v >= n) {
        if (per) { v -= n; shift = len; } else { valid = false; v = c; }
    }
    return v;
}

// Circular bodies of a DP update (Sec. 2.5), passed to kernels by value.
// A body of a DP update (Sec. 2.5): a circle of radius R about (cx, cy), or
// (sdf != NULL) SDF samples sdf[j * nx + i] at (ox, oy) + (i, j) h in the
// body's local frame, placed at (cx, cy) with posture angle theta
// (ct = cos theta, st = sin theta).  omega / omega_dot: angular velocity and
// acceleration (boundary velocity and Neumann datum).
struct BodyDev {
    int id;
    int nx, ny;
    double cx, cy, R;
    double ct, st;
    const double *sdf;
    double ox, oy, h;
    double omega, omega_dot;
};

// The bodies of one update, passed by value as a kernel parameter, with the
// weights Z (5 x 9) of the chi = 1 quadratic fit over a 3x3 lattice in units
// of its spacing (cos^2 weight, r_e = 2.5 spacings), shared by every SDF grid.
struct Bodies {
    int n;
    double Z[45];
    BodyDev c[MCD_MAX_BODIES];
};

// Circle SDF psi = |x - c| - R with every operation rounded on its own.
__device__ __forceinline__ double circle_psi(double x, double y, const BodyDev &b) {
    const double dx = __dsub_rn(x, b.cx);
    const double dy = __dsub_rn(y, b.cy);
    return __dsub_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))), b.R);
}

// psi and the world-frame grad psi of an SDF-grid body: the chi = 1
// quadratic fit centred at the grid point nearest the point (clamped so that
// its 3x3 support lies in the grid), evaluated at the point.  psi = +inf and
// grad = 0 outside the box of grid points 1 .. n - 2.
__device__ inline double sdf_eval(const BodyDev &b, const double *Z, double x, double y, double *gx, double *gy) {
    const double dx = __dsub_rn(x, b.cx), dy = __dsub_rn(y, b.cy);
    const double xl = __dadd_rn(__dmul_rn(b.ct, dx), __dmul_rn(b.st, dy));
    const double yl = __dadd_rn(__dmul_rn(-b.st, dx), __dmul_rn(b.ct, dy));
    const double fx = __ddiv_rn(__dsub_rn(xl, b.ox), b.h);
    const double fy = __ddiv_rn(__dsub_rn(yl, b.oy), b.h);
    *gx = 0.0;
    *gy = 0.0;
    if (!(fx >= 1.0 && fx <= (double)(b.nx - 2) && fy >= 1.0 && fy <= (double)(b.ny - 2))) return INFINITY;
    int i = (int)floor(fx + 0.5), j = (int)floor(fy + 0.5);
    i = i < 1 ? 1 : (i > b.nx - 2 ? b.nx - 2 : i);
    j = j < 1 ? 1 : (j > b.ny - 2 ? b.ny - 2 : j);
    const double ps = b.sdf[(int64_t)j * b.nx + i];
    double d[9];
#pragma unroll
    for (int s = 0; s < 9; ++s)
        d[s] = __dsub_rn(b.sdf[(int64_t)(j + s / 3 - 1) * b.nx + (i + s % 3 - 1)], ps);
    double Phi[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < 9; ++s) acc = __dadd_rn(acc, __dmul_rn(Z[q * 9 + s], d[s]));
        Phi[q] = acc;
    }
    const double X = __dsub_rn(fx, (double)i), Y = __dsub_rn(fy, (double)j);
    const double psi = ps + Phi[0] * X + Phi[1] * Y + 0.5 * Phi[2] * X * X + Phi[3] * X * Y + 0.5 * Phi[4] * Y * Y;
    const double gxl = (Phi[0] + Phi[2] * X + Phi[3] * Y) / b.h;
    const double gyl = (Phi[1] + Phi[3] * X + Phi[4] * Y) / b.h;
    *gx = b.ct * gxl - b.st * gyl;
    *gy = b.st * gxl + b.ct * gyl;
    return psi;
}

// SDF value of body b at (x, y).
__device__ __forceinline__ double body_psi(const Bodies &B, const BodyDev &b, double x, double y) {
    if (!b.sdf) return circle_psi(x, y, b);
    double gx, gy;
    return sdf_eval(b, B.Z, x, y, &gx, &gy);
}

// psi of body b at (x, y) and the unit vector along grad psi (false if it
// is undefined: the point at a circle's centre, outside an SDF grid, or a
// vanishing gradient).  Circles: the analytic (x - c) / |x - c|.
__device__ inline bool body_psi_dir(const Bodies &B, const BodyDev &b, double x, double y, double *psi,
                                    double *ux, double *uy) {
    if (!b.sdf) {
        const double dx = x - b.cx, dy = y - b.cy;
        const double d = sqrt(dx * dx + dy * dy);
        *psi = d - b.R;
        if (!(d > 0.0)) return false;
        *ux = dx / d;
        *uy = dy / d;
        return true;
    }
    double gx, gy;
    *psi = sdf_eval(b, B.Z, x, y, &gx, &gy);
    const double g = sqrt(gx * gx + gy * gy);
    if (!(g > 0.0) || !isfinite(*psi)) return false;
    *ux = gx / g;
    *uy = gy / g;
    return true;
}

// Index of the body whose SDF has the smallest magnitude at (x, y), the
// first on a tie (Sec. 2.5); its SDF value in *psi.
__device__ __forceinline__ int nearest_body(const Bodies &B, double x, double y, double *psi) {
    int best = 0;
    double bp = body_psi(B, B.c[0], x, y);
    for (int b = 1; b < B.n; ++b) {
        const double p = body_psi(B, B.c[b], x, y);
        if (fabs(p) < fabs(bp)) { best = b; bp = p; }
    }
    *psi = bp;
    return best;
}

__device__ __forceinline__ int body_with_id(const Bodies &B, int id) {
    for (int b = 0; b < B.n; ++b)
        if (B.c[b].id == id) return b;
    return -1;
}

// Checks a body list (2D mesh, 1..MCD_MAX_BODIES bodies, distinct ids in
// 2..127, positive radii of circles, SDF grids of at least 3 x 3 points
// with a positive spacing) and packs it for the kernels (update.cu).
mcd_status pack_bodies(const char *who, const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                       Bodies *out);

// Add n to the launch counter (launches made by a CUDA graph replay).
void count_launches(long long n);

// Solver workspace attached to a stencil handle (allocated on first solve).
struct Workspace;

// Scope guard around kernel launches: counts them and, when sampling is on,
// brackets the launch with CUDA events on its stream (mcd_timing_*).
class KTimer {
public:
    KTimer(int kind, cudaStream_t s, int nlaunch = 1);
    ~KTimer();
    KTimer(const KTimer &) = delete;
    KTimer &operator=(const KTimer &) = delete;

private:
    int kind_;
    cudaStream_t stream_;
    bool active_;
    cudaEvent_t a_{}, b_{};
};

}  // namespace mcd

struct mcd_stencils {
    mcd_mesh mesh;
    mcd_mls_params prm;
    mcd::Geo geo;
    int S;               // (2 support + 1)^dim: 9, 27 or 81
    int support;         // support radius R: 1 (3x3, 3x3x3) or 4 (2D 9x9)
    int shape;           // Shape<G> code G: 2, 3 or 9
    int nb;              // 5 or 9 derivative components
    int has_neumann;     // any bc_kind entry is Neumann
    double *row64;       // [S][N]
    float *row32;        // [S][N] (MIXED)
    double *ql64;        // [S][N] (has_neumann)
    double *d64;         // [nb][S][N] (want_derivs)
    double *qd64;        // [nb][S][N] (want_derivs && has_neumann)
    double *rscale;      // [N]
    int8_t *kind;        // [N]
    uint16_t *off16;     // [N][2] bf16 DP offsets (x - x_cell) / l0 (2D; network features)
    unsigned long long *bad_dp;  // device: smallest failing DP, ~0ull if none
    int *spmv_err;       // device: nonzero if a TMA-streamed SpMV gave up waiting for its copies
    mcd::Workspace *ws;
};

namespace mcd {
// Fill st->off16 from the DP positions (cnn.cu; no-op in 3D).
cudaError_t cnn_store_offsets(const mcd_stencils *st, const double *pos, const int8_t *mask,
                              cudaStream_t stream);
// Network warm start of a solve: p <- p + s e on the assembled system (cnn.cu).
mcd_status net_warm_start(const mcd_net *net, const mcd_stencils *st, const double *b,
                          const double *dprev, double *p, double *host_sc, cudaStream_t stream);
// Save the guess of a solve / write its increment p - guess (cnn.cu).
mcd_status net_save_guess(const mcd_net *net, const mcd_stencils *st, const double *p, cudaStream_t stream);
mcd_status net_store_increment(const mcd_net *net, const mcd_stencils *st, const double *p, double *dprev,
                               cudaStream_t stream);
}  // namespace mcd

namespace mcd {
// Batched stencil build over systems stored back to back (stencils.cu):
// system i has geometry geo[i], DP offset off[i] and its 128-thread blocks
// start at blk_start[i]; r_e and r_s of prm are multiples of each l0.
struct BatchBuildDesc {
    const Geo *geo;
    const int64_t *off;
    const int *blk_start;
    int nsys, nblocks;
    const double *pos;
    const int8_t *mask;
    const mcd_mls_params *prm;
    double *row64;
    float *row32;
    double *rscale;
    int8_t *kind;
    unsigned long long *bad;
};
cudaError_t launch_build_batch(const BatchBuildDesc &d, cudaStream_t stream);
}  // namespace mcd

// Launch a kernel inside a KTimer scope: MCD_KLAUNCH(kind, stream, k<<<...>>>(...));
#define MCD_KLAUNCH(kind, stream, ...)               \
    do {                                             \
        ::mcd::KTimer kt_launch_((kind), (stream));  \
        __VA_ARGS__;                                 \
    } while (0)

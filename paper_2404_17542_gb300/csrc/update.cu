// Moving-boundary DP update (arXiv 2404.17542, Sec. 2.2-2.4, Sec. 4.7).
//
// remask_kernel  one thread per cell: role reassignment inside the band from
//                the count of cell vertices with SDF >= 0 (Eq. (1)).  The
//                vertex test and the band test use explicitly rounded FP64
//                operations (__dmul_rn / __dadd_rn / __dsqrt_rn), so no
//                multiply-add is fused and the decision is bit-identical to
//                a plain IEEE evaluation of the same expression.
//                With several bodies each point takes the SDF of smallest
//                magnitude (Sec. 2.5; the first body on a tie), and a
//                boundary cell the id of the body nearest its centroid.
// relax_kernel   one thread per cell: one Jacobi sweep of spring relaxation
//                (Eqs. (5)-(8)), relocation onto the body (Eq. (9)),
//                optional boundary-fitted inner move (Eqs. (45)-(46)) and the
//                clamp into the cell; positions ping-pong between two buffers.
#include <math.h>

#include <cmath>

#include <mutex>

#include "common.cuh"

namespace mcd {

// Vertex (i, j) has psi >= 0 for its nearest body (tested as d^2 >= R^2).
__device__ __forceinline__ bool vertex_fluid(double ox, double oy, double l0, int i, int j, const Bodies &B) {
    const double vx = __dadd_rn(ox, __dmul_rn((double)i, l0));
    const double vy = __dadd_rn(oy, __dmul_rn((double)j, l0));
    double psi;
    const BodyDev &b = B.c[B.n > 1 ? nearest_body(B, vx, vy, &psi) : 0];
    if (b.sdf) return body_psi(B, b, vx, vy) >= 0.0;
    const double dx = __dsub_rn(vx, b.cx);
    const double dy = __dsub_rn(vy, b.cy);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return d2 >= __dmul_rn(b.R, b.R);
}

// Band test of cell (i, j) and (out) the index of the body nearest its
// centroid.
__device__ __forceinline__ bool cell_in_band(double ox, double oy, double l0, int i, int j,
                                             const Bodies &B, double band, int *nearest) {
    const double cx = __dadd_rn(ox, __dmul_rn((double)i + 0.5, l0));
    const double cy = __dadd_rn(oy, __dmul_rn((double)j + 0.5, l0));
    double psi;
    *nearest = nearest_body(B, cx, cy, &psi);
    if (band <= 0.0) return true;
    return fabs(psi) < band;
}

__global__ void remask_kernel(Geo g, Bodies bodies, double band, double *__restrict__ pos,
                              int8_t *__restrict__ mask, int8_t *__restrict__ mask_prev) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.N) return;
    const int nx = g.n[0], ny = g.n[1];
    const int i = (int)(k % nx), j = (int)(k / nx);
    const int8_t old = mask[k];
    mask_prev[k] = old;
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) return;   // wall cell
    int near = 0;
    if (!cell_in_band(g.org[0], g.org[1], g.l0, i, j, bodies, band, &near)) return;
    const int cnt = (int)vertex_fluid(g.org[0], g.org[1], g.l0, i, j, bodies) +
                    (int)vertex_fluid(g.org[0], g.org[1], g.l0, i + 1, j, bodies) +
                    (int)vertex_fluid(g.org[0], g.org[1], g.l0, i, j + 1, bodies) +
                    (int)vertex_fluid(g.org[0], g.org[1], g.l0, i + 1, j + 1, bodies);
    const int8_t nm = (cnt <= 1) ? (int8_t)0 : (cnt <= 3 ? (int8_t)bodies.c[near].id : (int8_t)-1);
    mask[k] = nm;
    if (nm == 0 && old != 0) {
        pos[k] = g.org[0] + ((double)i + 0.5) * g.l0;
        pos[g.N + k] = g.org[1] + ((double)j + 0.5) * g.l0;
    }
}

__global__ void relax_kernel(Geo g, Bodies bodies, double band, double kappa, double alpha,
                             const int8_t *__restrict__ mask, const double *__restrict__ pin,
                             double *__restrict__ pout) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.N;
    if (k >= N) return;
    const int nx = g.n[0], ny = g.n[1];
    const int i = (int)(k % nx), j = (int)(k / nx);
    const double xi = pin[k], yi = pin[N + k];
    const int8_t mk = mask[k];
    int near = 0;
    const bool movable = !(i == 0 || j == 0 || i == nx - 1 || j == ny - 1) && mk != 0 &&
                         cell_in_band(g.org[0], g.org[1], g.l0, i, j, bodies, band, &near);
    if (!movable) {
        pout[k] = xi;
        pout[N + k] = yi;
        return;
    }
    const double l0 = g.l0;
    const double sq2l0 = sqrt(2.0) * l0;
    double fx = 0.0, fy = 0.0;
    for (int dj = -1; dj <= 1; ++dj) {
        for (int di = -1; di <= 1; ++di) {
            if (di == 0 && dj == 0) continue;
            const int ii = i + di, jj = j + dj;
            if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
            const int64_t kk = (int64_t)ii + (int64_t)nx * jj;
            if (mask[kk] == 0) continue;
            const double ex = pin[kk] - xi, ey = pin[N + kk] - yi;      // x_ij = x_j - x_i
            const double r = sqrt(ex * ex + ey * ey);
            if (r == 0.0) continue;
            const double lspg = (di != 0 && dj != 0) ? sq2l0 : l0;       // Eq. (7)
            const double G = 1.0 - r / lspg;                            // Eq. (6)
            fx += G * (ex / r);                                         // Eq. (5)
            fy += G * (ey / r);
        }
    }
    double sx = xi - kappa * l0 * fx;                                   // Eq. (8)
    double sy = yi - kappa * l0 * fy;
    // a boundary DP follows its own body, an inner DP the nearest one
    int b = -1;
    if (mk >= 1) {
        b = body_with_id(bodies, mk);
    } else if (mk == -1 && alpha > 0.0) {
        double psi_near;
        b = bodies.n > 1 ? nearest_body(bodies, sx, sy, &psi_near) : 0;
    }
    double psi = 0.0, ux = 0.0, uy = 0.0;
    if (b >= 0 && body_psi_dir(bodies, bodies.c[b], sx, sy, &psi, &ux, &uy)) {
        const double hx = -ux, hy = -uy;                                // -grad psi / |grad psi|
        if (mk >= 1) {
            sx += psi * hx;                                             // Eq. (9)
            sy += psi * hy;
        } else {
            const double re = 5.0 * l0;
            if (psi < re) {
                const double beta = 0.5 * alpha * (1.0 + cos(M_PI * psi / re));   // Eq. (46)
                sx += beta * psi * hx;                                  // Eq. (45)
                sy += beta * psi * hy;
            }
        }
    }
    const double lox = g.org[0] + i * l0, loy = g.org[1] + j * l0;
    const double hix = g.org[0] + (i + 1) * l0, hiy = g.org[1] + (j + 1) * l0;
    pout[k] = fmin(fmax(sx, lox), hix);
    pout[N + k] = fmin(fmax(sy, loy), hiy);
}

// One 2D vector per body (accelerations or velocities), in body order.
struct BodyAcc {
    double a[MCD_MAX_BODIES][2];
};

__global__ void body_bc_kernel(Geo g, Bodies bodies, BodyAcc acc, const double *__restrict__ pos,
                               const int8_t *__restrict__ mask, double *__restrict__ nrm,
                               double *__restrict__ neu) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.N;
    if (k >= N) return;
    double nx = 0.0, ny = 0.0, ax = 0.0, ay = 0.0;
    const int b = mask[k] >= 1 ? body_with_id(bodies, mask[k]) : -1;
    if (b >= 0) {
        const BodyDev &body = bodies.c[b];
        double psi, ux, uy;
        if (body_psi_dir(bodies, body, pos[k], pos[N + k], &psi, &ux, &uy)) { nx = ux; ny = uy; }
        // dV/dt of a rigid body at x (Eqs. (26)-(29)): dV_trans/dt
        // + domega/dt x r + omega x (omega x r), r = x - x_c
        const double rx = pos[k] - body.cx, ry = pos[N + k] - body.cy;
        const double w2 = body.omega * body.omega;
        ax = acc.a[b][0] - body.omega_dot * ry - w2 * rx;
        ay = acc.a[b][1] + body.omega_dot * rx - w2 * ry;
    }
    nrm[k] = nx;
    nrm[N + k] = ny;
    if (neu) neu[k] = -(ax * nx + ay * ny);                            // Eq. (23)
}

// Boundary velocity of every DP: that of the rigid body whose id it carries
// at the DP's position, 0 elsewhere.
__global__ void body_vel_kernel(int64_t N, Bodies bodies, BodyAcc vel, const double *__restrict__ pos,
                                const int8_t *__restrict__ mask, double *__restrict__ ubc,
                                double *__restrict__ vbc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int b = mask[k] >= 1 ? body_with_id(bodies, mask[k]) : -1;
    if (b < 0) {
        ubc[k] = 0.0;
        vbc[k] = 0.0;
        return;
    }
    // V = V_trans + omega x r (Eqs. (24)-(25)), r = x - x_c
    const BodyDev &body = bodies.c[b];
    ubc[k] = vel.a[b][0] - body.omega * (pos[N + k] - body.cy);
    vbc[k] = vel.a[b][1] + body.omega * (pos[k] - body.cx);
}

// Checks the body list of an update and packs it for the kernels.
// Weights Z (5 x 9, slot s = (di+1) + 3 (dj+1)) of the chi = 1 quadratic fit
// over a 3x3 lattice in units of its spacing, cos^2 weight with r_e = 2.5
// (Eqs. (12)-(17)).  On the symmetric lattice the normal equations
// decouple: psi_X = sum w X dpsi / sum w X^2 (likewise psi_Y), psi_XY =
// sum w X Y dpsi / sum w X^2 Y^2, and a 2 x 2 system [[a, b], [b, a]] for
// psi_XX, psi_YY with a = sum w X^4 / 4, b = sum w X^2 Y^2 / 4.
static void sdf_fit_weights(double *Z) {
    const double re = 2.5;
    const double ca = std::cos(M_PI * 1.0 / (2.0 * re)), cd = std::cos(M_PI * std::sqrt(2.0) / (2.0 * re));
    const double wa = ca * ca, wd = cd * cd;
    const double a = (2.0 * wa + 4.0 * wd) / 4.0, bb = wd;
    for (int q = 0; q < 45; ++q) Z[q] = 0.0;
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            if (di == 0 && dj == 0) continue;
            const int s = (di + 1) + 3 * (dj + 1);
            const double w = (di == 0 || dj == 0) ? wa : wd;
            Z[0 * 9 + s] = w * di / (2.0 * wa + 4.0 * wd);
            Z[1 * 9 + s] = w * dj / (2.0 * wa + 4.0 * wd);
            Z[3 * 9 + s] = w * di * dj / (4.0 * wd);
            const double r1 = w * di * di / 2.0, r3 = w * dj * dj / 2.0;
            Z[2 * 9 + s] = (a * r1 - bb * r3) / (a * a - bb * bb);
            Z[4 * 9 + s] = (a * r3 - bb * r1) / (a * a - bb * bb);
        }
}

mcd_status pack_bodies(const char *who, const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                              Bodies *out) {
    if (mesh->dim != 2) {
        set_error(std::string(who) + ": 2D only");
        return MCD_ENOTSUP;
    }
    if (nbodies < 1 || nbodies > MCD_MAX_BODIES) {
        set_error(std::string(who) + ": nbodies must be in 1..MCD_MAX_BODIES");
        return MCD_EINVAL;
    }
    out->n = nbodies;
    for (int b = 0; b < nbodies; ++b) {
        if (bodies[b].id < 2 || bodies[b].id > 127) {
            set_error(std::string(who) + ": body id must be in 2..127");
            return MCD_EINVAL;
        }
        const mcd_body &bd = bodies[b];
        if (!bd.sdf_dev && !(bd.radius > 0.0)) {
            set_error(std::string(who) + ": a circle's radius must be positive");
            return MCD_EINVAL;
        }
        if (bd.sdf_dev && (bd.sdf_n[0] < 3 || bd.sdf_n[1] < 3 || !(bd.sdf_h > 0.0))) {
            set_error(std::string(who) + ": an SDF grid needs at least 3 x 3 points and a positive spacing");
            return MCD_EINVAL;
        }
        for (int a = 0; a < b; ++a)
            if (bodies[a].id == bodies[b].id) {
                set_error(std::string(who) + ": body ids must be distinct");
                return MCD_EINVAL;
            }
        BodyDev &o = out->c[b];
        o.id = bd.id;
        o.nx = bd.sdf_n[0];
        o.ny = bd.sdf_n[1];
        o.cx = bd.c[0];
        o.cy = bd.c[1];
        o.R = bd.radius;
        o.ct = std::cos(bd.theta);
        o.st = std::sin(bd.theta);
        o.sdf = bd.sdf_dev;
        o.ox = bd.sdf_origin[0];
        o.oy = bd.sdf_origin[1];
        o.h = bd.sdf_h;
        o.omega = bd.omega;
        o.omega_dot = bd.omega_dot;
    }
    sdf_fit_weights(out->Z);
    return MCD_OK;
}

// Position scratch for the Jacobi ping-pong, grown on demand and kept for
// the life of the process (one per device ordinal).
struct Scratch {
    double *buf = nullptr;
    size_t cap = 0;
};
static std::mutex g_scratch_mu;
static Scratch g_scratch[64];

static double *scratch_positions(size_t count) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    Scratch &s = g_scratch[dev];
    if (s.cap < count) {
        cudaFree(s.buf);
        s.buf = nullptr;
        s.cap = 0;
        if (cudaMalloc(&s.buf, count * sizeof(double)) != cudaSuccess) return nullptr;
        s.cap = count;
    }
    return s.buf;
}

}  // namespace mcd

using namespace mcd;

extern "C" mcd_status mcd_update_dps(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                                     double *pos_dev, int8_t *mask_dev, int8_t *mask_prev_dev,
                                     double kappa, int n_relax, double band, double alpha,
                                     mcd_stream_t stream) {
    MCD_CHECK_ARG(mesh && bodies && pos_dev && mask_dev && mask_prev_dev, "NULL argument");
    Bodies bl;
    mcd_status st = pack_bodies("mcd_update_dps", mesh, bodies, nbodies, &bl);
    if (st != MCD_OK) return st;
    MCD_CHECK_ARG(mesh->n[0] >= 3 && mesh->n[1] >= 3 && mesh->l0 > 0.0, "bad mesh");
    MCD_CHECK_ARG(n_relax >= 0 && kappa >= 0.0, "bad relaxation parameters");
    const Geo g = make_geo(*mesh);
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.N + threads - 1) / threads);
    MCD_KLAUNCH(MCD_K_UPDATE, stream, remask_kernel<<<blocks, threads, 0, stream>>>(g, bl, band, pos_dev, mask_dev, mask_prev_dev));
    MCD_LAUNCH_CHECK();
    if (n_relax == 0) return MCD_OK;
    double *tmp = scratch_positions(2 * (size_t)g.N);
    if (!tmp) {
        set_error("mcd_update_dps: scratch allocation failed");
        return MCD_ENOMEM;
    }
    double *a = pos_dev, *b = tmp;
    for (int it = 0; it < n_relax; ++it) {
        MCD_KLAUNCH(MCD_K_UPDATE, stream, relax_kernel<<<blocks, threads, 0, stream>>>(g, bl, band, kappa, alpha, mask_dev, a, b));
        double *t = a; a = b; b = t;
    }
    MCD_LAUNCH_CHECK();
    if (a != pos_dev)
        MCD_CUDA_TRY(cudaMemcpyAsync(pos_dev, a, 2 * (size_t)g.N * sizeof(double),
                                     cudaMemcpyDeviceToDevice, stream));
    return MCD_OK;
}

extern "C" mcd_status mcd_bodies_boundary(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                                          const double *pos_dev, const int8_t *mask_dev, double *normal_dev,
                                          double *neumann_dev, mcd_stream_t stream) {
    MCD_CHECK_ARG(mesh && bodies && pos_dev && mask_dev && normal_dev, "NULL argument");
    Bodies bl;
    mcd_status st = pack_bodies("mcd_bodies_boundary", mesh, bodies, nbodies, &bl);
    if (st != MCD_OK) return st;
    BodyAcc acc;
    for (int b = 0; b < nbodies; ++b) {
        acc.a[b][0] = bodies[b].acc[0];
        acc.a[b][1] = bodies[b].acc[1];
    }
    const Geo g = make_geo(*mesh);
    const unsigned blocks = (unsigned)((g.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, body_bc_kernel<<<blocks, 256, 0, stream>>>(g, bl, acc, pos_dev, mask_dev,
                                                                              normal_dev, neumann_dev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

extern "C" mcd_status mcd_bodies_velocity(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                                          const double *pos_dev, const int8_t *mask_dev, double *ubc_dev,
                                          double *vbc_dev, mcd_stream_t stream) {
    MCD_CHECK_ARG(mesh && bodies && pos_dev && mask_dev && ubc_dev && vbc_dev, "NULL argument");
    Bodies bl;
    mcd_status st = pack_bodies("mcd_bodies_velocity", mesh, bodies, nbodies, &bl);
    if (st != MCD_OK) return st;
    BodyAcc vel;
    for (int b = 0; b < nbodies; ++b) {
        vel.a[b][0] = bodies[b].vel[0];
        vel.a[b][1] = bodies[b].vel[1];
    }
    const Geo g = make_geo(*mesh);
    const unsigned blocks = (unsigned)((g.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, body_vel_kernel<<<blocks, 256, 0, stream>>>(g.N, bl, vel, pos_dev, mask_dev, ubc_dev,
                                                                               vbc_dev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

extern "C" mcd_status mcd_body_boundary(const mcd_mesh *mesh, const mcd_body *body, const double *pos_dev,
                                        const int8_t *mask_dev, double *normal_dev, double *neumann_dev,
                                        mcd_stream_t stream) {
    MCD_CHECK_ARG(body, "NULL argument");
    return mcd_bodies_boundary(mesh, body, 1, pos_dev, mask_dev, normal_dev, neumann_dev, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free DP update.
//
// Same computation as mcd_update_dps, but the Jacobi ping-pong positions live
// in the fixed device array below instead of memory obtained with cudaMalloc.
// It serves callers that must not allocate GPU memory while they step: a
// framework whose caching allocator has already reserved the device's memory,
// a time-stepping loop that cannot afford the device-wide synchronisation and
// unbounded latency that cudaMalloc / cudaFree can bring, or a code base that
// forbids allocation after start-up.  The array exists once per device that
// loads this library and stays reserved until the process exits.
// ---------------------------------------------------------------------------
namespace mcd {

static __device__ __align__(256) double g_noalloc_pos[2 * (size_t)MCD_NOALLOC_MAX_DPS];

static std::mutex g_noalloc_mu;
static double *g_noalloc_addr[64];   // device address of g_noalloc_pos, per device

// Device address of the fixed array on the current device.  The host-side
// symbol g_noalloc_pos is only a stand-in and must never reach a kernel; the
// real address is looked up once per device, with that device current.
static mcd_status noalloc_scratch(double **out) {
    int dev = 0;
    MCD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("mcd_update_dps_static: device ordinal out of range");
        return MCD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_pos);
        if (e != cudaSuccess || !p) {
            set_error(std::string("mcd_update_dps_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return MCD_ECUDA;
        }
        g_noalloc_addr[dev] = (double *)p;
    }
    *out = g_noalloc_addr[dev];
    return MCD_OK;
}

}  // namespace mcd

extern "C" mcd_status mcd_update_dps_static(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                                            double *pos_dev, int8_t *mask_dev, int8_t *mask_prev_dev,
                                            double kappa, int n_relax, double band, double alpha,
                                            mcd_stream_t stream) {
    MCD_CHECK_ARG(mesh && bodies && pos_dev && mask_dev && mask_prev_dev, "NULL argument");
    Bodies bl;
    mcd_status st = pack_bodies("mcd_update_dps_static", mesh, bodies, nbodies, &bl);
    if (st != MCD_OK) return st;
    MCD_CHECK_ARG(mesh->n[0] >= 3 && mesh->n[1] >= 3 && mesh->l0 > 0.0, "bad mesh");
    MCD_CHECK_ARG(n_relax >= 0 && kappa >= 0.0, "bad relaxation parameters");
    const Geo g = make_geo(*mesh);
    if (g.N > (int64_t)MCD_NOALLOC_MAX_DPS) {
        set_error("mcd_update_dps_static: mesh has " + std::to_string(g.N) +
                  " DPs, more than the fixed scratch holds (MCD_NOALLOC_MAX_DPS = " +
                  std::to_string((long long)MCD_NOALLOC_MAX_DPS) + ")");
        return MCD_EINVAL;
    }
    double *tmp = nullptr;
    st = noalloc_scratch(&tmp);
    if (st != MCD_OK) return st;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.N + threads - 1) / threads);
    MCD_KLAUNCH(MCD_K_UPDATE, stream, remask_kernel<<<blocks, threads, 0, stream>>>(g, bl, band, pos_dev, mask_dev,
                                                                                  mask_prev_dev));
    MCD_LAUNCH_CHECK();
    // Each sweep writes every one of the 2N scratch positions before any is
    // read, so contents left by an earlier call never leak into this one.
    double *a = pos_dev, *b = tmp;
    for (int it = 0; it < n_relax; ++it) {
        MCD_KLAUNCH(MCD_K_UPDATE, stream, relax_kernel<<<blocks, threads, 0, stream>>>(g, bl, band, kappa, alpha,
                                                                                     mask_dev, a, b));
        double *t = a; a = b; b = t;
    }
    MCD_LAUNCH_CHECK();
    if (a != pos_dev)
        MCD_CUDA_TRY(cudaMemcpyAsync(pos_dev, a, 2 * (size_t)g.N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     stream));
    return MCD_OK;
}

// ALE velocity interpolation and fluid force on a body (arXiv 2404.17542,
// Sec. 3.3 Eq. (19) and Appendix A; Sec. 3.4 Eqs. (30)-(31)).
//
// ale_kernel    one thread per DP: the step-k velocity at the DP's step-(k+1)
//               position, u~ = second-order Taylor value of the chi=1
//               quadratic MLS fit of the step-k cloud (Eq. (19), p = 2).  A DP
//               that moved into the fluid takes the fit of the DP at the
//               centre of its support shifted by one cell along the signs of
//               the nearest body's normal (Eq. (A.2)).
// force_kernel  one thread per DP over a fixed grid: the traction
//               t = (-P I + mu (grad u + grad u^T)) . n of each DP of the body,
//               with P and grad u from the fit of the shifted-support centre,
//               times the surface element (Eq. (31)); per-block partial sums,
//               then one block adds them in block order (deterministic).
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace mcd {

constexpr int ALE_S = 9;   // 3x3 stencils

// Global index of slot s of cell (ci, cj) (periodic wrap as in the build; an
// empty slot maps to the DP itself, whose weight there is 0).
__device__ __forceinline__ int64_t ale_slot_index(const Geo &g, int ci, int cj, int s, int64_t self) {
    bool valid = true;
    double sh;
    const int i = nb_coord(ci, s % 3 - 1, g.n[0], g.per[0], g.len[0], sh, valid);
    const int j = nb_coord(cj, s / 3 - 1, g.n[1], g.per[1], g.len[1], sh, valid);
    return valid ? (int64_t)i + (int64_t)g.n[0] * j : self;
}

// Physical derivatives (phi_x, phi_y, phi_xx, phi_xy, phi_yy) of a field at
// DP k from the derivative weights w [5][9][N] (and, if qw != NULL, the
// Neumann-data weights qw [5][9][N] applied to f).
__device__ __forceinline__ void fit_derivatives(const Geo &g, const double *__restrict__ w,
                                                const double *__restrict__ phi, const double *__restrict__ qw,
                                                const double *__restrict__ f, int64_t k, double *d) {
    const int64_t N = g.N;
    const int ci = (int)(k % g.n[0]), cj = (int)(k / g.n[0]);
    int64_t j[ALE_S];
#pragma unroll
    for (int s = 0; s < ALE_S; ++s) j[s] = ale_slot_index(g, ci, cj, s, k);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < ALE_S; ++s) acc += w[((int64_t)q * ALE_S + s) * N + k] * phi[j[s]];
        if (qw) {
#pragma unroll
            for (int s = 0; s < ALE_S; ++s) acc += qw[((int64_t)q * ALE_S + s) * N + k] * f[j[s]];
        }
        d[q] = acc;
    }
}

__device__ __forceinline__ double taylor2(double phi, const double *d, double dx, double dy) {
    return phi + dx * d[0] + dy * d[1] + 0.5 * (dx * dx * d[2] + 2.0 * dx * dy * d[3] + dy * dy * d[4]);
}

__device__ __forceinline__ int sgn(double v) { return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0); }

// Cell of the centre of DP k's support shifted by (sgn nx, sgn ny), clamped.
__device__ __forceinline__ int64_t shifted_centre(const Geo &g, int64_t k, int sx, int sy) {
    int i = (int)(k % g.n[0]) + sx, j = (int)(k / g.n[0]) + sy;
    i = i < 0 ? 0 : (i >= g.n[0] ? g.n[0] - 1 : i);
    j = j < 0 ? 0 : (j >= g.n[1] ? g.n[1] - 1 : j);
    return (int64_t)i + (int64_t)g.n[0] * j;
}

struct AleArgs {
    Geo g;
    const double *d64;      // step-k velocity derivative weights [5][9][N]
    const double *pos_k, *pos_k1;
    const int8_t *mask_k, *mask_k1;
    const double *u, *v;
    double *uo, *vo;
    int *fallbacks;         // device counter or NULL
    Bodies bodies;          // at step k
};

__global__ void __launch_bounds__(256) ale_kernel(const __grid_constant__ AleArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = a.g.N;
    if (k >= N) return;
    a.uo[k] = a.u[k];
    a.vo[k] = a.v[k];
    if (a.mask_k1[k] != -1) return;
    int64_t src = k;
    if (a.mask_k[k] != -1) {
        // moved into the fluid: the support shifted along the body normal
        const double x = a.pos_k[k], y = a.pos_k[N + k];
        double psi, ux = 0.0, uy = 0.0;
        const BodyDev &b = a.bodies.c[nearest_body(a.bodies, x, y, &psi)];
        if (!body_psi_dir(a.bodies, b, x, y, &psi, &ux, &uy)) { ux = 0.0; uy = 0.0; }
        src = shifted_centre(a.g, k, sgn(ux), sgn(uy));               // Eq. (A.2)
        if (a.mask_k[src] != -1) {
            if (a.fallbacks) atomicAdd(a.fallbacks, 1);
            return;
        }
    }
    const double dx = a.pos_k1[k] - a.pos_k[src];
    const double dy = a.pos_k1[N + k] - a.pos_k[N + src];
    double du[5], dv[5];
    fit_derivatives(a.g, a.d64, a.u, nullptr, nullptr, src, du);
    fit_derivatives(a.g, a.d64, a.v, nullptr, nullptr, src, dv);
    a.uo[k] = taylor2(a.u[src], du, dx, dy);                          // Eq. (19), (A.1)
    a.vo[k] = taylor2(a.v[src], dv, dx, dy);
}

constexpr int FORCE_BLOCKS = 304;   // 2 x 152 SMs; a grid-stride loop covers any N

struct ForceArgs {
    Geo g;
    const double *pd64, *pqd64, *bnd;   // pressure derivative / Neumann weights, boundary data
    const double *vd64;                 // velocity derivative weights
    const double *pos;
    const int8_t *mask;
    const double *normal;
    const double *P, *u, *v;
    double mu;
    int body_id;
    double *partials;                   // [3][FORCE_BLOCKS]
    int *skipped;
};

__global__ void __launch_bounds__(256) force_kernel(const __grid_constant__ ForceArgs a) {
    const int64_t N = a.g.N;
    const int nx = a.g.n[0], ny = a.g.n[1];
    double acc[3] = {0.0, 0.0, 0.0};   // Fx, Fy, sum dGamma
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        if (a.mask[k] != a.body_id) continue;
        const double nxk = a.normal[k], nyk = a.normal[N + k];
        const double xk = a.pos[k], yk = a.pos[N + k];
        // the nearest DP of the same boundary on each side of the tangent
        const double tx = -nyk, ty = nxk;
        double dpos = INFINITY, dneg = INFINITY;
        const int ci = (int)(k % nx), cj = (int)(k / nx);
        for (int dj = -2; dj <= 2; ++dj)
            for (int di = -2; di <= 2; ++di) {
                const int ii = ci + di, jj = cj + dj;
                if ((di == 0 && dj == 0) || ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
                const int64_t q = (int64_t)ii + (int64_t)nx * jj;
                if (a.mask[q] != a.body_id) continue;
                // separately rounded: the choice of neighbour is a decision
                const double ex = __dsub_rn(a.pos[q], xk), ey = __dsub_rn(a.pos[N + q], yk);
                const double side = __dadd_rn(__dmul_rn(ex, tx), __dmul_rn(ey, ty));
                if (side == 0.0) continue;
                const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
                if (side > 0.0) dpos = fmin(dpos, d); else dneg = fmin(dneg, d);
            }
        const double dG = 0.5 * ((isinf(dpos) ? 0.0 : dpos) + (isinf(dneg) ? 0.0 : dneg));   // Eq. (31)
        acc[2] += dG;
        const int64_t c = shifted_centre(a.g, k, sgn(nxk), sgn(nyk));
        if (a.mask[c] != -1) {
            atomicAdd(a.skipped, 1);
            continue;
        }
        const double dx = xk - a.pos[c], dy = yk - a.pos[N + c];
        double dP[5], du[5], dv[5];
        fit_derivatives(a.g, a.pd64, a.P, a.pqd64, a.bnd, c, dP);
        fit_derivatives(a.g, a.vd64, a.u, nullptr, nullptr, c, du);
        fit_derivatives(a.g, a.vd64, a.v, nullptr, nullptr, c, dv);
        const double Pk = taylor2(a.P[c], dP, dx, dy);
        const double ux = du[0] + du[2] * dx + du[3] * dy, uy = du[1] + du[3] * dx + du[4] * dy;
        const double vx = dv[0] + dv[2] * dx + dv[3] * dy, vy = dv[1] + dv[3] * dx + dv[4] * dy;
        const double trx = -Pk * nxk + a.mu * (2.0 * ux * nxk + (uy + vx) * nyk);
        const double try_ = -Pk * nyk + a.mu * ((uy + vx) * nxk + 2.0 * vy * nyk);
        acc[0] += trx * dG;                                            // Eq. (30)
        acc[1] += try_ * dG;
    }
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double x = acc[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < 8; ++w) x += red[threadIdx.x][w];
        a.partials[threadIdx.x * FORCE_BLOCKS + blockIdx.x] = x;
    }
}

// out[0..2] = sums of the partials in block order; out[3] = skipped DPs.
__global__ void force_sum_kernel(const double *__restrict__ partials, const int *__restrict__ skipped,
                                 double *__restrict__ out) {
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int b = 0; b < FORCE_BLOCKS; ++b) x += partials[threadIdx.x * FORCE_BLOCKS + b];
        out[threadIdx.x] = x;
    }
    if (threadIdx.x == 3) out[3] = (double)*skipped;
}

// Scratch of the force reduction: partials, the skipped counter, the result
// (one set per device ordinal, kept for the life of the process).
struct ForceScratch {
    double *partials = nullptr;
    int *skipped = nullptr;
    double *out = nullptr;
};
static std::mutex g_force_mu;
static ForceScratch g_force[64];

static mcd_status force_scratch(ForceScratch **out) {
    int dev = 0;
    MCD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("mcd_fluid_force: device ordinal out of range");
        return MCD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_force_mu);
    ForceScratch &s = g_force[dev];
    if (!s.partials) {
        if (cudaMalloc(&s.partials, 3 * FORCE_BLOCKS * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s.skipped, sizeof(int)) != cudaSuccess || cudaMalloc(&s.out, 4 * sizeof(double)) != cudaSuccess) {
            cudaFree(s.partials);
            cudaFree(s.skipped);
            cudaFree(s.out);
            s = ForceScratch();
            set_error("mcd_fluid_force: scratch allocation failed");
            return MCD_ENOMEM;
        }
    }
    *out = &s;
    return MCD_OK;
}

static mcd_status check_derivs(const mcd_stencils *st, const char *who) {
    MCD_CHECK_ARG(st, "NULL stencil handle");
    if (st->mesh.dim != 2 || st->support != 1) {
        set_error(std::string(who) + ": 2D 3x3 stencils only");
        return MCD_ENOTSUP;
    }
    MCD_CHECK_ARG(st->d64, "the stencil handle needs want_derivs = 1");
    return MCD_OK;
}

}  // namespace mcd

using namespace mcd;

extern "C" mcd_status mcd_ale_interpolate(const mcd_stencils *vel_k, const mcd_body *bodies_k, int nbodies,
                                          const double *pos_k_dev, const double *pos_k1_dev,
                                          const int8_t *mask_k_dev, const int8_t *mask_k1_dev,
                                          const double *u_dev, const double *v_dev, double *u_out_dev,
                                          double *v_out_dev, int *fallbacks_dev, mcd_stream_t stream) {
    mcd_status st = check_derivs(vel_k, "mcd_ale_interpolate");
    if (st != MCD_OK) return st;
    MCD_CHECK_ARG(bodies_k && pos_k_dev && pos_k1_dev && mask_k_dev && mask_k1_dev && u_dev && v_dev &&
                      u_out_dev && v_out_dev,
                  "NULL argument");
    MCD_CHECK_ARG(u_out_dev != u_dev && v_out_dev != v_dev && u_out_dev != v_dev && v_out_dev != u_dev,
                  "outputs must not alias the step-k fields");
    AleArgs a;
    st = pack_bodies("mcd_ale_interpolate", &vel_k->mesh, bodies_k, nbodies, &a.bodies);
    if (st != MCD_OK) return st;
    a.g = vel_k->geo;
    a.d64 = vel_k->d64;
    a.pos_k = pos_k_dev;
    a.pos_k1 = pos_k1_dev;
    a.mask_k = mask_k_dev;
    a.mask_k1 = mask_k1_dev;
    a.u = u_dev;
    a.v = v_dev;
    a.uo = u_out_dev;
    a.vo = v_out_dev;
    a.fallbacks = fallbacks_dev;
    const unsigned blocks = (unsigned)((a.g.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, ale_kernel<<<blocks, 256, 0, stream>>>(a));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

extern "C" mcd_status mcd_fluid_force(const mcd_stencils *pres, const mcd_stencils *vel, int body_id,
                                      const double *pos_dev, const int8_t *mask_dev, const double *normal_dev,
                                      const double *P_dev, const double *bnd_dev, const double *u_dev,
                                      const double *v_dev, double mu, double *out_host, mcd_stream_t stream) {
    mcd_status st = check_derivs(pres, "mcd_fluid_force");
    if (st != MCD_OK) return st;
    st = check_derivs(vel, "mcd_fluid_force");
    if (st != MCD_OK) return st;
    MCD_CHECK_ARG(pres->geo.N == vel->geo.N && pres->mesh.n[0] == vel->mesh.n[0], "handles of different meshes");
    MCD_CHECK_ARG(pos_dev && mask_dev && normal_dev && P_dev && u_dev && v_dev && out_host, "NULL argument");
    MCD_CHECK_ARG(!pres->qd64 || bnd_dev, "the pressure handle has Neumann ids: bnd is required");
    MCD_CHECK_ARG(body_id >= 1 && body_id <= 127, "body id must be in 1..127");
    ForceScratch *sc = nullptr;
    st = force_scratch(&sc);
    if (st != MCD_OK) return st;
    ForceArgs a;
    a.g = pres->geo;
    a.pd64 = pres->d64;
    a.pqd64 = pres->qd64;
    a.bnd = bnd_dev;
    a.vd64 = vel->d64;
    a.pos = pos_dev;
    a.mask = mask_dev;
    a.normal = normal_dev;
    a.P = P_dev;
    a.u = u_dev;
    a.v = v_dev;
    a.mu = mu;
    a.body_id = body_id;
    a.partials = sc->partials;
    a.skipped = sc->skipped;
    MCD_CUDA_TRY(cudaMemsetAsync(sc->skipped, 0, sizeof(int), stream));
    MCD_KLAUNCH(MCD_K_OTHER, stream, force_kernel<<<FORCE_BLOCKS, 256, 0, stream>>>(a));
    MCD_KLAUNCH(MCD_K_OTHER, stream, force_sum_kernel<<<1, 32, 0, stream>>>(sc->partials, sc->skipped, sc->out));
    MCD_LAUNCH_CHECK();
    MCD_CUDA_TRY(cudaMemcpyAsync(out_host, sc->out, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MCD_CUDA_TRY(cudaStreamSynchronize(stream));
    return MCD_OK;
}

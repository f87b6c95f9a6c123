// Fractional-step driver around the pressure solve (arXiv 2404.17542,
// Sec. 3.3, Eqs. (20)-(22)), 2D, FP64, one thread per DP.
//
// flow_predict_kernel  u* = F_MOC + nu dt lap u: the departure value at
//                      x - u dt from the DP's second-order Taylor expansion
//                      (gradient and Hessian from the MLS derivative weights,
//                      Eq. (14)), plus the viscous term; boundary DPs take the
//                      prescribed velocity, void DPs 0.
// flow_div_kernel      (1/dt) div u* at inner DPs (the PPE source, Eq. (21)).
// flow_project_kernel  u = u* - dt grad P (Eq. (22)); grad P includes the
//                      Neumann-data terms of the MLS fit (Eq. (15)).
#include "common.cuh"

namespace mcd {

// Derivatives (nb = 5: x, y, xx, xy, yy) of a field at DP k from the value
// weights d64 [5][9][N].
__device__ __forceinline__ void derivs5(const double *__restrict__ d64, const double *__restrict__ phi,
                                        const int64_t *nb, int64_t N, int64_t k, double *out) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int s = 0; s < 9; ++s) acc += d64[((int64_t)c * 9 + s) * N + k] * phi[nb[s]];
        out[c] = acc;
    }
}

__device__ __forceinline__ void neighbours9(const Geo &g, int64_t k, int64_t *nb) {
    const int i = (int)(k % g.n[0]), j = (int)(k / g.n[0]);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int ii = i + s % 3 - 1, jj = j + s / 3 - 1;
        if (ii < 0) ii = g.per[0] ? ii + g.n[0] : i;
        if (ii >= g.n[0]) ii = g.per[0] ? ii - g.n[0] : i;
        if (jj < 0) jj = g.per[1] ? jj + g.n[1] : j;
        if (jj >= g.n[1]) jj = g.per[1] ? jj - g.n[1] : j;
        nb[s] = (int64_t)ii + (int64_t)g.n[0] * jj;
    }
}

__global__ void flow_predict_kernel(Geo g, const int8_t *__restrict__ kind, const double *__restrict__ d64,
                                    const double *__restrict__ u, const double *__restrict__ v,
                                    const double *__restrict__ ubc, const double *__restrict__ vbc,
                                    double nu, double dt, double *__restrict__ us, double *__restrict__ vs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.N;
    if (k >= N) return;
    const int8_t kd = kind[k];
    if (kd != KIND_INNER) {
        us[k] = (kd == KIND_VOID) ? 0.0 : ubc[k];
        vs[k] = (kd == KIND_VOID) ? 0.0 : vbc[k];
        return;
    }
    int64_t nb[9];
    neighbours9(g, k, nb);
    double du[5], dv[5];
    derivs5(d64, u, nb, N, k, du);
    derivs5(d64, v, nb, N, k, dv);
    const double uk = u[k], vk = v[k];
    const double dx = -uk * dt, dy = -vk * dt;
    const double mu = uk + dx * du[0] + dy * du[1] + 0.5 * (dx * dx * du[2] + 2.0 * dx * dy * du[3] + dy * dy * du[4]);
    const double mv = vk + dx * dv[0] + dy * dv[1] + 0.5 * (dx * dx * dv[2] + 2.0 * dx * dy * dv[3] + dy * dy * dv[4]);
    us[k] = mu + nu * dt * (du[2] + du[4]);
    vs[k] = mv + nu * dt * (dv[2] + dv[4]);
}

__global__ void flow_div_kernel(Geo g, const int8_t *__restrict__ kind, const double *__restrict__ d64,
                                const double *__restrict__ us, const double *__restrict__ vs, double dt,
                                double *__restrict__ src) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.N;
    if (k >= N) return;
    if (kind[k] != KIND_INNER) { src[k] = 0.0; return; }
    int64_t nb[9];
    neighbours9(g, k, nb);
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        ax += d64[((int64_t)0 * 9 + s) * N + k] * us[nb[s]];
        ay += d64[((int64_t)1 * 9 + s) * N + k] * vs[nb[s]];
    }
    src[k] = (ax + ay) / dt;
}

__global__ void flow_project_kernel(Geo g, const int8_t *__restrict__ kind, const double *__restrict__ d64,
                                    const double *__restrict__ qd64, const double *__restrict__ P,
                                    const double *__restrict__ bnd, const double *__restrict__ us,
                                    const double *__restrict__ vs, const double *__restrict__ ubc,
                                    const double *__restrict__ vbc, double dt, double *__restrict__ u,
                                    double *__restrict__ v) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.N;
    if (k >= N) return;
    const int8_t kd = kind[k];
    if (kd != KIND_INNER) {
        u[k] = (kd == KIND_VOID) ? 0.0 : ubc[k];
        v[k] = (kd == KIND_VOID) ? 0.0 : vbc[k];
        return;
    }
    int64_t nb[9];
    neighbours9(g, k, nb);
    double px = 0.0, py = 0.0;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const double pj = P[nb[s]];
        px += d64[((int64_t)0 * 9 + s) * N + k] * pj;
        py += d64[((int64_t)1 * 9 + s) * N + k] * pj;
        if (qd64) {
            const double fj = bnd[nb[s]];
            px += qd64[((int64_t)0 * 9 + s) * N + k] * fj;
            py += qd64[((int64_t)1 * 9 + s) * N + k] * fj;
        }
    }
    u[k] = us[k] - dt * px;
    v[k] = vs[k] - dt * py;
}

}  // namespace mcd

using namespace mcd;

static mcd_status flow_check(const mcd_stencils *st) {
    MCD_CHECK_ARG(st, "NULL handle");
    if (st->mesh.dim != 2 || st->support != 1) {
        set_error("flow driver: 2D 3x3 stencils only");
        return MCD_ENOTSUP;
    }
    MCD_CHECK_ARG(st->d64, "flow driver needs a stencil handle built with want_derivs = 1");
    return MCD_OK;
}

extern "C" mcd_status mcd_flow_predict(const mcd_stencils *vel, const double *u_dev, const double *v_dev,
                                       const double *ubc_dev, const double *vbc_dev, double nu, double dt,
                                       double *us_dev, double *vs_dev, double *src_dev, mcd_stream_t stream) {
    mcd_status s = flow_check(vel);
    if (s != MCD_OK) return s;
    MCD_CHECK_ARG(u_dev && v_dev && ubc_dev && vbc_dev && us_dev && vs_dev && src_dev, "NULL argument");
    MCD_CHECK_ARG(dt > 0.0 && nu >= 0.0, "dt must be positive and nu non-negative");
    MCD_CHECK_ARG(us_dev != u_dev && vs_dev != v_dev, "u* must not alias u");
    const unsigned blocks = (unsigned)((vel->geo.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, flow_predict_kernel<<<blocks, 256, 0, stream>>>(
                                         vel->geo, vel->kind, vel->d64, u_dev, v_dev, ubc_dev, vbc_dev, nu, dt,
                                         us_dev, vs_dev));
    MCD_KLAUNCH(MCD_K_OTHER, stream, flow_div_kernel<<<blocks, 256, 0, stream>>>(vel->geo, vel->kind, vel->d64,
                                                                                 us_dev, vs_dev, dt, src_dev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

extern "C" mcd_status mcd_flow_project(const mcd_stencils *pst, const double *P_dev, const double *bnd_dev,
                                       const double *us_dev, const double *vs_dev, const double *ubc_dev,
                                       const double *vbc_dev, double dt, double *u_dev, double *v_dev,
                                       mcd_stream_t stream) {
    mcd_status s = flow_check(pst);
    if (s != MCD_OK) return s;
    MCD_CHECK_ARG(P_dev && bnd_dev && us_dev && vs_dev && ubc_dev && vbc_dev && u_dev && v_dev, "NULL argument");
    MCD_CHECK_ARG(dt > 0.0, "dt must be positive");
    const unsigned blocks = (unsigned)((pst->geo.N + 255) / 256);
    MCD_KLAUNCH(MCD_K_OTHER, stream, flow_project_kernel<<<blocks, 256, 0, stream>>>(
                                         pst->geo, pst->kind, pst->d64, pst->qd64, P_dev, bnd_dev, us_dev, vs_dev,
                                         ubc_dev, vbc_dev, dt, u_dev, v_dev));
    MCD_LAUNCH_CHECK();
    return MCD_OK;
}

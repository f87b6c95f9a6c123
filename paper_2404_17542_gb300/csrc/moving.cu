// One moving-boundary fractional step (arXiv 2404.17542, Sec. 3.3) behind
// the C ABI: the library sequences the stages of the step and forms the
// rigid-body accelerations of the Neumann datum itself, so that a C caller
// runs the paper's step with one call per time step.
//
// Order of a step (Sec. 3.3; Sec. 2.3-2.4 for the DP update, Appendix A for
// the ALE fill, Sec. 3.4 for the force):
//   1. dV/dt and d omega/dt of every body by the finite differences of
//      Eq. (29) between the step-k and step-(k+1) body states;
//   2. DP update to the step-(k+1) bodies (remask, relaxation, relocation);
//   3. ALE interpolation of u and v (and optionally of P, the PPE's initial
//      guess) to the new positions (Eq. (19), Appendix A Eqs. (A.1)-(A.2))
//      with the step-k velocity stencils;
//   4. velocity stencils of the new cloud (every boundary a value boundary),
//      body normals and Neumann data dP/dn = -dV/dt . n (Eq. (23)), pressure
//      stencils (bodies Neumann, walls Dirichlet);
//   5. boundary velocities V + omega x r (Eqs. (24)-(25)), u* and the PPE
//      source (Eqs. (20)-(21));
//   6. the PPE solve (Sec. 3.3), the projection u = u* - dt grad P (Eq. (22));
//   7. the fluid force on every body (Eqs. (30)-(31)), mu = nu.
// Every stage is one of the library's own entry points; this file only
// allocates the step's work arrays and calls them in order.
#include <string.h>

#include <cmath>

#include "common.cuh"

struct mcd_flow {
    mcd_mesh mesh;
    mcd_flow_params prm;
    int64_t N = 0;
    int nbodies = 0;
    int ids[MCD_MAX_BODIES];
    mcd_stencils *vel = nullptr;    // velocity stencils of the current cloud
    mcd_stencils *pres = nullptr;   // pressure stencils of the current cloud
    double *pos_k = nullptr;        // [2][N] step-k positions
    int8_t *mask_k = nullptr, *mask_prev = nullptr;
    double *ut = nullptr, *vt = nullptr, *us = nullptr, *vs = nullptr, *src = nullptr;
    double *ubc = nullptr, *vbc = nullptr, *normal = nullptr, *bnd = nullptr, *b = nullptr;
    double *guess = nullptr, *scratch = nullptr;
    int *fallbacks = nullptr;       // device counters: [0] velocity ALE, [1] pressure ALE
};

namespace mcd {
namespace {

void free_flow(mcd_flow *f) {
    if (!f) return;
    if (f->vel) mcd_stencils_destroy(f->vel);
    if (f->pres) mcd_stencils_destroy(f->pres);
    cudaFree(f->pos_k); cudaFree(f->mask_k); cudaFree(f->mask_prev);
    cudaFree(f->ut); cudaFree(f->vt); cudaFree(f->us); cudaFree(f->vs); cudaFree(f->src);
    cudaFree(f->ubc); cudaFree(f->vbc); cudaFree(f->normal); cudaFree(f->bnd); cudaFree(f->b);
    cudaFree(f->guess); cudaFree(f->scratch); cudaFree(f->fallbacks);
    delete f;
}

mcd_mls_params mls_params(const mcd_flow *f, int pressure) {
    mcd_mls_params p;
    memset(&p, 0, sizeof(p));
    p.weight_kind = f->prm.weight_kind;
    p.r_e = f->prm.r_e > 0.0 ? f->prm.r_e : f->mesh.l0;
    p.r_s = f->mesh.l0;
    p.precision = pressure ? f->prm.precision : MCD_FP64;
    p.want_derivs = 1;
    p.support = 1;
    if (pressure)
        for (int b = 0; b < f->nbodies; ++b) p.bc_kind[f->ids[b]] = MCD_BC_NEUMANN;
    return p;
}

// The step-(k+1) bodies with the accelerations of Eq. (29): the finite
// differences of the translational and angular velocities over the step.
mcd_status differenced_bodies(const mcd_flow *f, const mcd_body *bk, const mcd_body *b1, int nbodies,
                              double dt, mcd_body *out) {
    MCD_CHECK_ARG(nbodies == f->nbodies, "the body list changed length since mcd_flow_create");
    for (int i = 0; i < nbodies; ++i) {
        MCD_CHECK_ARG(bk[i].id == f->ids[i] && b1[i].id == f->ids[i],
                      "body ids must match those given to mcd_flow_create, in the same order");
        out[i] = b1[i];
        for (int d = 0; d < 3; ++d) out[i].acc[d] = (b1[i].vel[d] - bk[i].vel[d]) / dt;
        out[i].omega_dot = (b1[i].omega - bk[i].omega) / dt;
    }
    return MCD_OK;
}

}  // namespace
}  // namespace mcd

using namespace mcd;

#define FLOW_TRY(call)                         \
    do {                                       \
        mcd_status s_ = (call);                \
        if (s_ != MCD_OK) return s_;           \
    } while (0)

extern "C" mcd_status mcd_flow_create(const mcd_mesh *mesh, const mcd_flow_params *prm,
                                      const mcd_body *bodies, int nbodies, double *pos_dev,
                                      int8_t *mask_dev, mcd_flow **out, mcd_stream_t stream) {
    MCD_CHECK_ARG(mesh && prm && bodies && pos_dev && mask_dev && out, "NULL argument");
    MCD_CHECK_ARG(mesh->dim == 2, "the moving-boundary step is 2D (MCD_ENOTSUP otherwise)");
    MCD_CHECK_ARG(nbodies >= 1 && nbodies <= MCD_MAX_BODIES, "nbodies must be in 1..MCD_MAX_BODIES");
    MCD_CHECK_ARG(prm->nu >= 0.0 && std::isfinite(prm->nu), "nu must be finite and >= 0");
    MCD_CHECK_ARG(prm->precision == MCD_FP64 || prm->precision == MCD_MIXED, "unknown precision");
    MCD_CHECK_ARG(prm->n_relax >= 0, "n_relax must be >= 0");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    mcd_flow *f = new mcd_flow();
    f->mesh = *mesh;
    f->prm = *prm;
    f->N = (int64_t)mesh->n[0] * mesh->n[1];
    f->nbodies = nbodies;
    for (int b = 0; b < nbodies; ++b) f->ids[b] = bodies[b].id;
    const size_t n8 = (size_t)f->N * sizeof(double);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void **)&f->pos_k, 2 * n8);
    alloc((void **)&f->mask_k, f->N);
    alloc((void **)&f->mask_prev, f->N);
    alloc((void **)&f->ut, n8); alloc((void **)&f->vt, n8);
    alloc((void **)&f->us, n8); alloc((void **)&f->vs, n8); alloc((void **)&f->src, n8);
    alloc((void **)&f->ubc, n8); alloc((void **)&f->vbc, n8);
    alloc((void **)&f->normal, 2 * n8); alloc((void **)&f->bnd, n8); alloc((void **)&f->b, n8);
    alloc((void **)&f->guess, n8); alloc((void **)&f->scratch, n8);
    alloc((void **)&f->fallbacks, 2 * sizeof(int));
    if (e != cudaSuccess) {
        free_flow(f);
        set_error(std::string("mcd_flow_create: ") + cudaGetErrorString(e));
        return MCD_ENOMEM;
    }
    // the first arrangement: every cell (band 0), as at the start of a run
    mcd_status s = mcd_update_dps(mesh, bodies, nbodies, pos_dev, mask_dev, f->mask_prev, prm->kappa,
                                  prm->n_relax, 0.0, prm->alpha, stream);
    if (s == MCD_OK) {
        const mcd_mls_params vp = mls_params(f, 0);
        s = mcd_build_stencils(mesh, pos_dev, mask_dev, nullptr, &vp, &f->vel, stream);
    }
    if (s == MCD_OK && cudaMemsetAsync(f->fallbacks, 0, 2 * sizeof(int), st) != cudaSuccess) s = MCD_ECUDA;
    if (s != MCD_OK) {
        free_flow(f);
        return s;
    }
    *out = f;
    return MCD_OK;
}

extern "C" void mcd_flow_destroy(mcd_flow *f) { free_flow(f); }

extern "C" mcd_status mcd_flow_restart(mcd_flow *f, const double *pos_dev, const int8_t *mask_dev,
                                       mcd_stream_t stream) {
    MCD_CHECK_ARG(f && pos_dev && mask_dev, "NULL argument");
    const mcd_mls_params vp = mls_params(f, 0);
    return mcd_build_stencils(&f->mesh, pos_dev, mask_dev, nullptr, &vp, &f->vel, stream);
}

extern "C" mcd_status mcd_flow_step(mcd_flow *f, const mcd_body *bodies_k, const mcd_body *bodies_k1,
                                    int nbodies, double dt, const mcd_solve_params *solve,
                                    double *pos_dev, int8_t *mask_dev, double *u_dev, double *v_dev,
                                    double *P_dev, mcd_flow_info *info, mcd_stream_t stream) {
    MCD_CHECK_ARG(f && bodies_k && bodies_k1 && solve && pos_dev && mask_dev && u_dev && v_dev && P_dev,
                  "NULL argument");
    MCD_CHECK_ARG(dt > 0.0 && std::isfinite(dt), "dt must be positive and finite");
    cudaStream_t st = (cudaStream_t)stream;
    const mcd_mesh *mesh = &f->mesh;
    const int64_t N = f->N;
    const size_t n8 = (size_t)N * sizeof(double);
    mcd_body b1[MCD_MAX_BODIES];
    FLOW_TRY(differenced_bodies(f, bodies_k, bodies_k1, nbodies, dt, b1));
    const double band = f->prm.band > 0.0 ? f->prm.band : 5.0 * mesh->l0;

    // 2. DP update (the step-k cloud is kept for the ALE interpolation)
    MCD_CUDA_TRY(cudaMemcpyAsync(f->pos_k, pos_dev, 2 * n8, cudaMemcpyDeviceToDevice, st));
    MCD_CUDA_TRY(cudaMemcpyAsync(f->mask_k, mask_dev, (size_t)N, cudaMemcpyDeviceToDevice, st));
    MCD_CUDA_TRY(cudaMemsetAsync(f->fallbacks, 0, 2 * sizeof(int), st));
    FLOW_TRY(mcd_update_dps(mesh, b1, nbodies, pos_dev, mask_dev, f->mask_prev, f->prm.kappa, f->prm.n_relax,
                            band, f->prm.alpha, stream));
    // 3. ALE interpolation with the step-k velocity stencils
    FLOW_TRY(mcd_ale_interpolate(f->vel, bodies_k, nbodies, f->pos_k, pos_dev, f->mask_k, mask_dev, u_dev, v_dev,
                                 f->ut, f->vt, f->fallbacks, stream));
    if (f->prm.ale_pressure) {
        FLOW_TRY(mcd_ale_interpolate(f->vel, bodies_k, nbodies, f->pos_k, pos_dev, f->mask_k, mask_dev, P_dev,
                                     P_dev, f->guess, f->scratch, f->fallbacks + 1, stream));
        MCD_CUDA_TRY(cudaMemcpyAsync(P_dev, f->guess, n8, cudaMemcpyDeviceToDevice, st));
    } else {
        MCD_CUDA_TRY(cudaMemcpyAsync(f->guess, P_dev, n8, cudaMemcpyDeviceToDevice, st));
    }
    // 4. stencils of the new cloud, normals and Neumann data
    const mcd_mls_params vp = mls_params(f, 0);
    FLOW_TRY(mcd_build_stencils(mesh, pos_dev, mask_dev, nullptr, &vp, &f->vel, stream));
    FLOW_TRY(mcd_bodies_boundary(mesh, b1, nbodies, pos_dev, mask_dev, f->normal, f->bnd, stream));
    const mcd_mls_params pp = mls_params(f, 1);
    FLOW_TRY(mcd_build_stencils(mesh, pos_dev, mask_dev, f->normal, &pp, &f->pres, stream));
    // 5. boundary velocities, u* and the PPE source
    FLOW_TRY(mcd_bodies_velocity(mesh, b1, nbodies, pos_dev, mask_dev, f->ubc, f->vbc, stream));
    FLOW_TRY(mcd_flow_predict(f->vel, f->ut, f->vt, f->ubc, f->vbc, f->prm.nu, dt, f->us, f->vs, f->src,
                              stream));
    FLOW_TRY(mcd_assemble_rhs(f->pres, f->src, f->bnd, f->b, stream));
    // 6. PPE and projection
    mcd_solve_info si;
    memset(&si, 0, sizeof(si));
    const mcd_status ss = mcd_solve_pressure(f->pres, f->src, f->bnd, P_dev, solve, &si, stream);
    if (info) {
        memset(info, 0, sizeof(*info));
        info->solve = si;
        info->nbodies = nbodies;
    }
    if (ss != MCD_OK) return ss;
    FLOW_TRY(mcd_flow_project(f->pres, P_dev, f->bnd, f->us, f->vs, f->ubc, f->vbc, dt, u_dev, v_dev, stream));
    // 7. forces (each call synchronises the stream)
    for (int b = 0; b < nbodies; ++b) {
        double F[4] = {0.0, 0.0, 0.0, 0.0};
        if (f->prm.forces)
            FLOW_TRY(mcd_fluid_force(f->pres, f->vel, f->ids[b], pos_dev, mask_dev, f->normal, P_dev, f->bnd,
                                     u_dev, v_dev, f->prm.nu, F, stream));
        if (info) {
            info->force[b][0] = F[0];
            info->force[b][1] = F[1];
            info->perimeter[b] = F[2];
            info->skipped[b] = (int)F[3];
        }
    }
    if (info) {
        int fb[2] = {0, 0};
        MCD_CUDA_TRY(cudaMemcpyAsync(fb, f->fallbacks, sizeof(fb), cudaMemcpyDeviceToHost, st));
        MCD_CUDA_TRY(cudaStreamSynchronize(st));
        info->ale_fallbacks = fb[0];
        info->ale_fallbacks_p = fb[1];
    }
    return MCD_OK;
}

extern "C" const mcd_stencils *mcd_flow_stencils(const mcd_flow *f, int which) {
    if (!f) return nullptr;
    return which == MCD_FLOW_PRESSURE ? f->pres : (which == MCD_FLOW_VELOCITY ? f->vel : nullptr);
}

extern "C" mcd_status mcd_flow_copy(const mcd_flow *f, int which, double *dst_dev, mcd_stream_t stream) {
    MCD_CHECK_ARG(f && dst_dev, "NULL argument");
    const double *src = nullptr;
    size_t n = (size_t)f->N;
    switch (which) {
    case MCD_FLOW_B: src = f->b; break;
    case MCD_FLOW_GUESS: src = f->guess; break;
    case MCD_FLOW_BND: src = f->bnd; break;
    case MCD_FLOW_SRC: src = f->src; break;
    case MCD_FLOW_NORMAL: src = f->normal; n *= 2; break;
    default: set_error("unknown flow array"); return MCD_EINVAL;
    }
    MCD_CUDA_TRY(cudaMemcpyAsync(dst_dev, src, n * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MCD_OK;
}

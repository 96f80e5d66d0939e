/*
 * glbm.h -- C ABI of the homogenised porous-medium LBM in liblbm.so.
 *
 * Sec. 4 of the paper compares the pore-scale solution with the generalised
 * lattice Boltzmann model (GLBM) of Guo & Zhao (2002): the volume-averaged
 * flow obeys Eqs. (GeneralizedPor1), (GeneralizedPor2) with the porous-medium
 * force of Eq. (PorousForce),
 *     F = -(eps nu / K) u - (eps c_F / sqrt(K)) |u| u + eps G,
 * with porosity eps, permeability K, Forchheimer coefficient c_F, effective
 * viscosity nu_eff = (tau - 1/2) / 3 and body force G.  The discrete scheme is
 * Guo & Zhao's: D3Q19 BGK with f_k^eq = w_k rho (1 + 3 e.u + 9/2 (e.u)^2/eps -
 * 3/2 u.u/eps), the source F_k = w_k rho (1 - 1/(2 tau)) (3 e.F + 9 (e.u)(e.F)
 * /eps - 3 u.F/eps), and u = v / (c0 + sqrt(c0^2 + c1 |v|)) with v = sum e f /
 * rho + eps G/2, c0 = (1 + eps nu/(2K))/2, c1 = eps c_F/(2 sqrt K).
 *
 * eps, 1/K and tau are given per z-plane (1/K = 0: free fluid; the paper's
 * proposed model takes nu_eff = nu/eps in the porous region, i.e. tau(z) =
 * 3 nu / eps(z) + 1/2).  The box is periodic in x and y.  Unless periodic_z,
 * the planes z = 0 and nz - 1 are walls with half-way bounce-back, a moving
 * wall adding -6 w_k rho (e_k . u_wall) to the returning population.
 *
 * Conventions are those of lbm.h: LBM_* status codes, caller-owned device
 * workspace (256-byte aligned), calls asynchronous on the bound stream unless
 * they return host values.  Populations are FP32, stored as f_k - w_k in place
 * (AA pattern), one slot per fluid cell and direction.
 */
#ifndef GLBM_H
#define GLBM_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glbm_solver glbm_solver;

typedef struct {
    int32_t nx, ny, nz;       /* box; fluid planes 1..nz-2, or 0..nz-1 if periodic_z */
    int32_t periodic_z;
    double nu;                /* viscosity in the Darcy term of Eq. (PorousForce) */
    double c_f;               /* Forchheimer coefficient */
    double g[3];              /* body force G */
    double u_bottom[3];       /* velocity of the wall z = 0 */
    double u_top[3];          /* velocity of the wall z = nz - 1 */
} glbm_params;

/* Workspace bytes for a box (LBM_EINVAL for a box below 1 x 1 x 3, or above
 * 2^31 fluid cells). */
int glbm_workspace_size(const glbm_params *params, size_t *bytes);

/* Bind the workspace, upload the per-plane tables eps[nz], inv_k[nz] (1/K)
 * and tau[nz] (host, FP64; tau > 1/2, 0 < eps <= 1, inv_k >= 0; wall planes
 * ignored) and initialise f = f^eq(rho = 1, u0) with dev_u0 [3][nz][ny][nx]
 * (float, may be NULL for rest).  Synchronises `stream`. */
int glbm_init(const glbm_params *params, const double *eps, const double *inv_k, const double *tau,
              void *dev_workspace, size_t bytes, const float *dev_u0, void *stream, glbm_solver **out);

/* n time steps (n >= 0). */
int glbm_step(glbm_solver *solver, int64_t n);

/* Density and velocity (Guo & Zhao's u) of the current state, dense
 * [nz][ny][nx] (dev_rho) and [3][nz][ny][nx] (dev_u); wall planes 0.  Either
 * pointer may be NULL. */
int glbm_moments(glbm_solver *solver, float *dev_rho, float *dev_u);

/* Plane averages of u_x, host_out[nz] (FP64 sums; wall planes 0).
 * Synchronises the stream. */
int glbm_plane_average(glbm_solver *solver, double *host_out);

/* The populations f_k - w_k of the current time, dev_out [19][n_fluid]
 * (fluid cells in order x fastest, then y, then z). */
int glbm_populations(glbm_solver *solver, float *dev_out);

/* Steps taken since glbm_init. */
int glbm_steps_done(const glbm_solver *solver, int64_t *steps);

void glbm_destroy(glbm_solver *solver);

#ifdef __cplusplus
}
#endif

#endif /* GLBM_H */

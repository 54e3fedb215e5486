/*
 * Drag gradient with respect to the shape of a fixed metaball: a hand-written
 * discrete adjoint of the lattice sweep (pull stream, BGK collision with Guo
 * forcing, §2.2 Eqs. (14)-(18)), of the velocity-interpolated bounce-back on
 * the particle links (§2.3.1 Eqs. (19)-(25), with the link fraction q of
 * Eq. (27)) and of the momentum-exchange force (§2.3.2 Eqs. (28)-(29)).
 *
 * Setting.  One fixed particle in a fully periodic box, FP32 populations
 * (offset form, as the main sweep), D3Q19.  The node flags are classified once
 * from the particle given to lbm_adj_init() and frozen: a forward run with
 * another geometry keeps the same links and only their q changes.  The
 * objective is the mean drag J = (1/W) sum_{t=T-W}^{T-1} F_x(t) over the last
 * W of T steps, starting from f^eq(rho0, u0).  The gradient is dJ/dK_i and
 * dJ/dx_i for every control point (weight K_i, world position x_i, Eq. (4)):
 * the adjoint runs backwards through the T steps, recomputing the states of
 * each segment of ceil(sqrt(T)) steps from a checkpoint kept by the forward
 * run, and accumulates dJ/dq per link, which the chain rule through Eq. (27)
 * and Eq. (4) turns into the shape gradient.  The paper has no adjoint.
 *
 * Memory: the caller owns one device workspace (lbm_adj_workspace_size, 256-
 * byte aligned), borrowed until lbm_adj_destroy(); the handle is a small host
 * allocation.  Work runs on the stream given to lbm_adj_init().  Errors: the
 * lbm_status codes of lbm_metaball.h; lbm_adj_last_error() gives a message.
 */
#ifndef LBM_ADJOINT_H
#define LBM_ADJOINT_H

#include "lbm_metaball.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_adj lbm_adj;

/* Device bytes for the configuration (nx, ny, nz, all three periodic[] = 1,
 * lattice 19, tau, rho0, c0, u0, force are read), the particle (its node
 * flags decide the link count), T >= 1 steps and 1 <= W <= T window steps. */
int lbm_adj_workspace_size(const lbm_config *cfg, const lbm_particle *p, int T, int W, size_t *bytes);

/* Classify the particle's nodes (frozen from now on) and build the links. */
int lbm_adj_init(const lbm_config *cfg, const lbm_particle *p, int T, int W, void *dev_ws, size_t ws_bytes,
                 void *cuda_stream, lbm_adj **out);

/* Forward run with control points at cp_world (host double[ncp][3], world
 * frame) with weights K (host double[ncp]), ncp as in the particle given to
 * lbm_adj_init; returns J (synchronises).  Keeps the checkpoints the
 * backward run needs. */
int lbm_adj_forward(lbm_adj *a, const double *cp_world, const double *K, double *J);

/* Gradient of the J of the last forward run: dJ_dcp host double[ncp][3],
 * dJ_dK host double[ncp] (either may be NULL).  Synchronises. */
int lbm_adj_backward(lbm_adj *a, double *dJ_dcp, double *dJ_dK);

/* Links (fluid node, direction) crossing the frozen surface, and the
 * checkpoint interval. */
int lbm_adj_info(const lbm_adj *a, int *nlinks, int *checkpoint_every);

int lbm_adj_destroy(lbm_adj *a);

const char *lbm_adj_last_error(const lbm_adj *a);

#ifdef __cplusplus
}
#endif
#endif

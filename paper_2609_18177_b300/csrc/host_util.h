// Host helpers shared by the entry points: problem validation and the
// translation of an lbmh_problem into the kernels' DevParams.
#pragma once
#include <math.h>

#include <cmath>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "../../include/lbmh.h"
#include "common.cuh"

namespace lbmh {

inline int nfields(int sys, int dim) {
  switch (sys) {
    case SYS_ADV: return 1;
    case SYS_EULER: return dim + 2;
    case SYS_SWE: return dim + 1;
    case SYS_REACT: return dim + 3;
  }
  return -1;
}

// reflecting or inflow sides, or a sponge: implemented by the fused kernels only
inline bool needs_fused(const lbmh_problem* p) {
  bool special = p->sponge_width > 0.0;
  for (int s = 0; s < 2 * p->dim; s++) special = special || p->bc[s] == LBMH_BC_REFLECT || p->bc[s] == LBMH_BC_INFLOW;
  return special;
}

inline int validate(const lbmh_problem* p, std::string& why) {
  if (!p) { why = "problem is NULL"; return LBMH_ERR_INVALID_ARG; }
  if (p->system == LBMH_LINEAR) { why = "LBMH_LINEAR is provided by the oracle only"; return LBMH_ERR_UNSUPPORTED; }
  if (p->system < 0 || p->system > 3) { why = "unknown system"; return LBMH_ERR_INVALID_ARG; }
  if (p->dim < 1 || p->dim > 3) { why = "dim must be 1, 2 or 3"; return LBMH_ERR_INVALID_ARG; }
  if (p->nx < 1 || (p->dim >= 2 && p->ny < 1) || (p->dim == 3 && p->nz < 1)) { why = "grid must have at least one node"; return LBMH_ERR_INVALID_ARG; }
  if ((long long)p->nx * (p->dim >= 2 ? p->ny : 1) * (p->dim == 3 ? p->nz : 1) > (1ll << 34)) { why = "grid too large"; return LBMH_ERR_INVALID_ARG; }
  if (p->dim == 3) {
    if (p->system == LBMH_SWE) { why = "3D lattices: advection, Euler and reactive Euler"; return LBMH_ERR_UNSUPPORTED; }
    for (int s = 0; s < 4; s++)
      if (p->bc[s] != LBMH_BC_PERIODIC && p->bc[s] != LBMH_BC_OUTFLOW) { why = "3D lattices: periodic or outflow sides"; return LBMH_ERR_UNSUPPORTED; }
    for (int s = 0; s < 2; s++)
      if (p->bc_z[s] != LBMH_BC_PERIODIC && p->bc_z[s] != LBMH_BC_OUTFLOW) { why = "3D lattices: periodic or outflow sides"; return LBMH_ERR_UNSUPPORTED; }
    if ((p->bc_z[0] == LBMH_BC_PERIODIC) != (p->bc_z[1] == LBMH_BC_PERIODIC)) { why = "periodic z boundaries must pair"; return LBMH_ERR_INVALID_ARG; }
    double dx = (p->x1 - p->x0) / p->nx, dz = (p->z1 - p->z0) / p->nz;
    if (!(fabs(dx - dz) <= 1e-12 * dx)) { why = "3D mesh must satisfy dx == dy == dz"; return LBMH_ERR_INVALID_ARG; }
    if (p->sponge_width != 0.0) { why = "no sponge on 3D lattices"; return LBMH_ERR_UNSUPPORTED; }
  }
  if (!(p->x1 > p->x0)) { why = "x1 must exceed x0"; return LBMH_ERR_INVALID_ARG; }
  for (int s = 0; s < 2 * p->dim; s++)
    if (p->bc[s] < LBMH_BC_PERIODIC || p->bc[s] > LBMH_BC_INFLOW) { why = "bad boundary condition"; return LBMH_ERR_INVALID_ARG; }
  for (int s = 0; s < 2 * p->dim; s++)
    if (p->bc[s] == LBMH_BC_REFLECT && (s < 2 ? p->nx : p->ny) < 4) {
      why = "a reflecting side needs at least 4 nodes across";
      return LBMH_ERR_INVALID_ARG;
    }
  if (!(p->sponge_width >= 0.0) || p->sponge_width > p->x1 - p->x0) { why = "sponge width must lie in [0, x1 - x0]"; return LBMH_ERR_INVALID_ARG; }
  for (int s = 0; s < 2 * p->dim; s++)
    if (p->bc[s] == LBMH_BC_INFLOW) {
      const double* u = p->u_in;
      bool ok = true;
      for (int c = 0; c < nfields(p->system, p->dim); c++) ok = ok && std::isfinite(u[c]);
      if (p->system == LBMH_SWE || p->system == LBMH_EULER || p->system == LBMH_REACTIVE_EULER) ok = ok && u[0] > 0.0;
      if (p->system == LBMH_EULER || p->system == LBMH_REACTIVE_EULER) {
        double msq = u[1] * u[1] + (p->dim == 2 ? u[2] * u[2] : 0.0);
        double chem = p->system == LBMH_REACTIVE_EULER ? p->q * u[p->dim + 2] : 0.0;
        ok = ok && (u[p->dim + 1] - 0.5 * msq / u[0] - chem) > 0.0;
      }
      if (!ok) { why = "u_in must be a finite physical state for an inflow side"; return LBMH_ERR_INVALID_ARG; }
    }
  if ((p->bc[0] == LBMH_BC_PERIODIC) != (p->bc[1] == LBMH_BC_PERIODIC)) { why = "periodic x boundaries must pair"; return LBMH_ERR_INVALID_ARG; }
  if (p->dim >= 2) {
    if ((p->bc[2] == LBMH_BC_PERIODIC) != (p->bc[3] == LBMH_BC_PERIODIC)) { why = "periodic y boundaries must pair"; return LBMH_ERR_INVALID_ARG; }
    double dx = (p->x1 - p->x0) / p->nx, dy = (p->y1 - p->y0) / p->ny;
    if (!(fabs(dx - dy) <= 1e-12 * dx)) { why = "2D mesh must satisfy dx == dy (Section 2.2.2)"; return LBMH_ERR_INVALID_ARG; }
  }
  if (!(p->cfl > 0.0)) { why = "cfl must be positive"; return LBMH_ERR_INVALID_ARG; }
  if (!(p->eps >= 0.0)) { why = "eps must be non-negative"; return LBMH_ERR_INVALID_ARG; }
  if (p->precision != LBMH_FP64 && p->precision != LBMH_FP32) { why = "bad precision"; return LBMH_ERR_INVALID_ARG; }
  if (p->kernel < 0 || p->kernel > 2) { why = "bad kernel choice"; return LBMH_ERR_INVALID_ARG; }
  if (p->omega_mode != 0 && p->omega_mode != 1) { why = "bad omega mode"; return LBMH_ERR_INVALID_ARG; }
  if ((p->system == LBMH_EULER || p->system == LBMH_REACTIVE_EULER) && !(p->gamma > 1.0)) { why = "gamma must exceed 1"; return LBMH_ERR_INVALID_ARG; }
  if (p->system == LBMH_SWE && !(p->g > 0.0)) { why = "g must be positive"; return LBMH_ERR_INVALID_ARG; }
  if (p->system == LBMH_SWE && p->bed_amp != 0.0 && !(p->bed_w2 > 0.0)) { why = "bed width must be positive"; return LBMH_ERR_INVALID_ARG; }
  return LBMH_OK;
}

// DevParams of a problem whose rows have the given pitch (elements)
inline DevParams make_devparams(const lbmh_problem* p, int pitch) {
  DevParams P;
  memset(&P, 0, sizeof P);
  P.nx = p->nx;
  P.ny3 = p->dim >= 2 ? p->ny : 1;
  P.nz3 = p->dim == 3 ? p->nz : 1;
  P.ny = P.ny3 * P.nz3;  // rows (z outer) in 3D
  P.pitch = pitch;
  P.plane = (long long)P.ny * P.pitch;
  P.ywin0 = 0;
  P.ywin1 = P.ny;
  P.row0 = 0;
  P.first_wait_polls = 1 << 22;
  for (int s = 0; s < 4; s++) P.bc[s] = p->bc[s];
  if (p->dim == 1) P.bc[2] = P.bc[3] = LBMH_BC_PERIODIC;
  P.bc_z[0] = p->dim == 3 ? p->bc_z[0] : LBMH_BC_PERIODIC;
  P.bc_z[1] = p->dim == 3 ? p->bc_z[1] : LBMH_BC_PERIODIC;
  P.x0 = p->x0;
  P.y0 = p->dim >= 2 ? p->y0 : 0.0;
  P.z0 = p->dim == 3 ? p->z0 : 0.0;
  P.adv_z = p->dim == 3 ? p->adv_z : 0.0;
  P.dx = (p->x1 - p->x0) / p->nx;
  P.cfl = p->cfl;
  P.eps = p->eps;
  P.T = 0.0;
  P.max_steps = 0;
  P.adv[0] = p->adv[0];
  P.adv[1] = p->adv[1];
  P.gamma = p->gamma;
  P.g = p->g;
  P.h_dry = p->h_dry > 0.0 ? p->h_dry : 1e-5;
  P.bed_amp = p->bed_amp;
  P.bed_w2 = p->bed_w2 > 0.0 ? p->bed_w2 : 1.0;
  P.bed_xc = p->bed_xc;
  P.bed_yc = p->bed_yc;
  P.K = p->K;
  P.Ti = p->Ti;
  P.q = p->q;
  P.has_bed = p->bed_amp != 0.0;
  P.has_react = p->K != 0.0;
  P.sponge_width = p->sponge_width;
  P.sponge_dx_over_w = p->sponge_width > 0.0 ? P.dx / p->sponge_width : 0.0;
  for (int c = 0; c < 8; c++) P.u_in[c] = p->u_in[c];
  P.has_special_bc = 0;
  for (int s = 0; s < 4; s++) P.has_special_bc |= (p->bc[s] == LBMH_BC_REFLECT || p->bc[s] == LBMH_BC_INFLOW);
  P.omega_mode = p->omega_mode;
  P.omega_fixed = p->omega_fixed;
  PhysConstF& f = P.pf;
  f.gamma = (float)P.gamma;
  f.gm1 = (float)(P.gamma - 1.0);
  f.g = (float)P.g;
  f.half_g = (float)(0.5 * P.g);
  f.h_dry = (float)P.h_dry;
  f.cmin = (float)sqrt(P.g * P.h_dry);
  f.q = (float)P.q;
  f.adv0 = (float)P.adv[0];
  f.adv1 = (float)P.adv[1];
  f.dx = (float)P.dx;
  f.bed_amp = (float)P.bed_amp;
  f.bed_inv_w2 = (float)(1.0 / P.bed_w2);
  f.bed_m2_inv_w2 = (float)(-2.0 / P.bed_w2);
  f.xb = (float)(P.x0 + 0.5 * P.dx - P.bed_xc);
  f.yb = (float)(P.y0 + 0.5 * P.dx - P.bed_yc);
  f.K = (float)P.K;
  f.Ti = (float)P.Ti;
  f.omega_fixed = (float)P.omega_fixed;
  f.adv2 = (float)P.adv_z;
  f.sponge_dx_over_w = (float)P.sponge_dx_over_w;
  for (int c = 0; c < 8; c++) f.u_in[c] = (float)P.u_in[c];
  return P;
}

// test hook: LBMH_TEST_FIRST_WAIT_POLLS sets the polls of each CTA's first
// row-load wait (0: the wait gives up at once and the step reports a timeout)
inline void apply_wait_hook(DevParams& P) {
  const char* e = getenv("LBMH_TEST_FIRST_WAIT_POLLS");
  if (e && e[0]) P.first_wait_polls = atoi(e);
}

// elements per row of a padded distribution plane (rows start on 128 bytes)
inline int padded_pitch(int nx, size_t elem) {
  int align = 128 / (int)elem;
  return (nx + 2 * XPAD + align - 1) / align * align;
}

}  // namespace lbmh

// State of the Poisson conjugate-gradient iteration (Section 2.3) shared by the launch-per-
// step iteration (fe_poisson.cu) and the persistent float iteration (fe_cg_fused.cu).
#pragma once

#include <cstdint>

#include "fe_internal.h"

namespace fe_cg {

// coarse functions per plane with the in-plane modes: the indicator, cos x, sin x, cos y,
// sin y, cos x cos y, cos x sin y, sin x cos y, sin x sin y
constexpr int MODES_NM = 9;

struct CgState {
  double rz, rz_new, pq, rr, alpha, beta, bnorm2, tol2, mean;
  int done, iters, maxit;
  unsigned int ticket[2];   // finished-block counters of the single-pass reductions (0 at rest)
  int fused_err;            // persistent iteration: a grid barrier gave up (0 at rest)
};

// Buffers of the float iteration with the plane coarse space (n_phi nodes, planes of a
// multiple of four nodes, 16-byte aligned vectors).
struct FusedCg {
  float *x, *r, *z, *p, *q;
  const float* dinv;
  const unsigned char* mask;
  const double* Ainv;   // nzp x nzp inverse of the coarse matrix
  const double* cnt;    // free nodes per plane
  CgState* s;
  int project;          // CEF: residuals are kept at zero mean
  // in-plane mode coarse space (nullptr: the plane indicators alone): the inverses of the
  // MODES_NM - 1 mode coarse matrices [MODES_NM - 1][nz][nz] (in the order above, float) and the
  // float mode tables (cos x, sin x [NX]; cos y, sin y [NY])
  const float* Amodes;
  const float* mtab;
};

// Early stop of a persistent launch: it returns after the first iteration whose float
// residual satisfies rr <= rr_lo or !(rr <= rr_hi), or that reaches iters_stop iterations
// (or convergence, or the iteration cap in the state).
struct FusedStop {
  double rr_lo, rr_hi;
  int iters_stop;
};

// true when the persistent iteration runs on this mesh (p = 1..6, a cooperative launch that
// fits the device, planes of a multiple of four nodes)
bool fused_available(fe_mesh* m);
// up to nit iterations in one cooperative launch on the mesh's stream (asynchronous); the
// state's fused_err reports a barrier that gave up
fe_status fused_run(fe_mesh* m, const FusedCg& b, int nit, const FusedStop& stop);

}  // namespace fe_cg

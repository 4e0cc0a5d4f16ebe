// Templated preconditioner pieces shared between trace_ops.cu and pressure_mg.cu.
#pragma once

#include "hmg_internal.cuh"

namespace hmg {

// One pressure-multigrid V-cycle for H_0 x = b from a zero initial guess (Sec. 2.3), in
// precision T (double: FP64 operator; float: the FP32 copies). b [ncell] in T. On return
// *x points at the level-0 work vector holding the result (valid until the next V-cycle).
// With x0, the finest level starts from x0 instead of zero (its first sweep smooths x0).
template <typename T>
int vcycle(Ctx *c, const T *b, T **x, const T *x0 = nullptr);

// The same V-cycle with b = Gamma P^T R (Algorithm 2 lines 4-5) computed inside its first
// sweep from the trace residual R [ntrace]; b is also stored in cb [ncell] (in T).
template <typename T>
int vcycle_trace(Ctx *c, const T *R, T *cb, T **x);

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const double *S(const Ctx *c) { return c->S; }
  static const double *Sz_w(const Ctx *c) { return c->Sz_w; }
  static const double *Sz_l(const Ctx *c) { return c->Sz_l; }
  static const double *Sz_cp(const Ctx *c) { return c->Sz_cp; }
  static const double *Sh_w(const Ctx *c) { return c->Sh_w; }
  static const double *gamma(const Ctx *c) { return c->gamma; }
  static const double *H(const Level &l) { return l.H; }
  static const double *Hz_w(const Level &l) { return l.Hz_w; }
  static const double *Hz_l(const Level &l) { return l.Hz_l; }
  static const double *Hz_cp(const Level &l) { return l.Hz_cp; }
};
template <>
struct Prec<float> {
  static const float *S(const Ctx *c) { return c->S32; }
  static const float *Sz_w(const Ctx *c) { return c->Sz_w32; }
  static const float *Sz_l(const Ctx *c) { return c->Sz_l32; }
  static const float *Sz_cp(const Ctx *c) { return c->Sz_cp32; }
  static const float *Sh_w(const Ctx *c) { return c->Sh_w32; }
  static const float *gamma(const Ctx *c) { return c->gamma32; }
  static const float *H(const Level &l) { return l.H32; }
  static const float *Hz_w(const Level &l) { return l.Hz_w32; }
  static const float *Hz_l(const Level &l) { return l.Hz_l32; }
  static const float *Hz_cp(const Level &l) { return l.Hz_cp32; }
};

}  // namespace hmg

// Exponential Runge-Kutta drivers around the phi-function actions (Sec. 2, Eq. (RK) with the
// Butcher tableaus of Table RK): exponential Euler, the two-stage method (c2 = 1/2) and the
// three-stage method (c2 = 1/3, c3 = 2/3), for u' + A u = f(u) with A a Kronecker sum.
//
// With D_j = f(U_j) - A u (A applied to the step's starting value u, as in Eq. (RK)):
//   Euler  u+ = u + tau phi_1(-tau A) D_1
//   RK2    U_2 = u + tau c2 phi_1(-c2 tau A) D_1
//          u+  = u + tau phi_1(-tau A) ((1 - 1/(2c2)) D_1 + 1/(2c2) D_2)
//   RK3    U_2 = u + tau c2 phi_1(-c2 tau A) D_1
//          U_3 = u + tau (2/3 phi_1(-c3 tau A) D_1 + 4/(9c2) phi_2(-c3 tau A) (D_2 - D_1))
//          u+  = u + tau (phi_1(-tau A) D_1 + 3/2 phi_2(-tau A) (D_3 - D_1))
// (the tableau rows regrouped by linearity: every phi-action of a stage shares one plan, and
// the two right-hand sides of a plan go through one phikron_apply_many call).
//
// One plan per distinct c_j tau (phi_0 skipped).  A u is applied from the nonzeros of the 1D
// factors (CSR per dimension) by one kernel; f(U) - A u and the stage combinations are
// elementwise float64 kernels (a few flops per unknown, HBM-bound).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "checked.cuh"
#include "common.h"
#include "profile.h"

PK_CHK_BIND(erk)

namespace phikron {
namespace {

constexpr int EW = 256;

struct Csr {
  const int* rowptr;
  const int* col;
  const double* val;
};

struct KronCsr {
  Csr f[PHIKRON_MAX_DIMS];
  int n[PHIKRON_MAX_DIMS];
  int dims;
};

// Au = sum_d (A^d acting on axis d) u, from the nonzeros of each factor
__global__ void __launch_bounds__(EW) kron_csr_kernel(KronCsr K, const double* __restrict__ u,
                                                     double* __restrict__ Au, long long N) {
  for (long long idx = blockIdx.x * (long long)EW + threadIdx.x; idx < N; idx += (long long)gridDim.x * EW) {
    double acc = 0.0;
    long long stride = 1;
    long long rest = idx;
    for (int d = K.dims - 1; d >= 0; --d) {
      const int nd = K.n[d];
      const int i = (int)(rest % nd);
      rest /= nd;
      const long long base = idx - (long long)i * stride;
      const Csr c = K.f[d];
      const int q0 = chk::ld_ck(c.rowptr + i, chk::SITE_ERK), q1 = chk::ld_ck(c.rowptr + i + 1, chk::SITE_ERK);
      for (int q = q0; q < q1; ++q)
        acc = fma(chk::ld_ck(c.val + q, chk::SITE_ERK),
                  chk::ld_ck(u + base + (long long)chk::ld_ck(c.col + q, chk::SITE_ERK) * stride, chk::SITE_ERK), acc);
      stride *= nd;
    }
    chk::st_ck(Au + idx, acc, chk::SITE_ERK);
  }
}

// D = f(U) - Au (- S if S is given)
__global__ void __launch_bounds__(EW) residual_kernel(int nonlin, const double* __restrict__ U,
                                                     const double* __restrict__ Au, const double* __restrict__ S,
                                                     double* __restrict__ D, long long N) {
  for (long long i = blockIdx.x * (long long)EW + threadIdx.x; i < N; i += (long long)gridDim.x * EW) {
    const double x = chk::ld_ck(U + i, chk::SITE_ERK);
    double f = 0.0;
    if (nonlin == PHIKRON_NONLIN_ALLEN_CAHN) f = x - x * x * x;
    double d = f - chk::ld_ck(Au + i, chk::SITE_ERK);
    if (S) d -= chk::ld_ck(S + i, chk::SITE_ERK);
    chk::st_ck(D + i, d, chk::SITE_ERK);
  }
}

// out = base + sum_{k < nx} c[k] X[k]  (out may alias base)
struct Comb {
  const double* X[3];
  double c[3];
  int nx;
};

__global__ void __launch_bounds__(EW) combine_kernel(const double* base, Comb cb, double* out, long long N) {
  for (long long i = blockIdx.x * (long long)EW + threadIdx.x; i < N; i += (long long)gridDim.x * EW) {
    double v = base ? chk::ld_ck(base + i, chk::SITE_ERK) : 0.0;
    for (int k = 0; k < cb.nx; ++k) v = fma(cb.c[k], chk::ld_ck(cb.X[k] + i, chk::SITE_ERK), v);
    chk::st_ck(out + i, v, chk::SITE_ERK);
  }
}

int ew_blocks(long long N) { return (int)std::max(1LL, std::min((N + EW - 1) / EW, 152LL * 8)); }

}  // namespace
}  // namespace phikron

using namespace phikron;

struct phikron_erk_s {
  phikron::Profiler prof;   // the integrator's own kernels (stencil, residual, stage combinations)
  int method = 0, dims = 0, nonlin = 0;
  int n[PHIKRON_MAX_DIMS] = {1, 1, 1, 1, 1, 1};
  long long N = 0;
  double tau = 0.0;
  int device = -1;
  // plans in the order the step uses them: Euler {1}; RK2 {c2, 1}; RK3 {c2, c3, 1}
  std::vector<phikron_plan_t> plans;
  std::vector<double> cs;
  std::vector<int> lmax;
  KronCsr K{};
  std::vector<void*> allocs;
  double *Au = nullptr, *D1 = nullptr, *D2 = nullptr, *D3 = nullptr, *U2 = nullptr, *V2 = nullptr, *Out = nullptr;
  ~phikron_erk_s() {
    for (phikron_plan_t p : plans) phikron_destroy(p);
    for (void* a : allocs) device_free(a);
  }
  int alloc(void** p, size_t bytes) {
    PK_RET(device_malloc(p, std::max<size_t>(bytes, 16), "phikron_erk_create"));
    allocs.push_back(*p);
    return PHIKRON_OK;
  }
};

namespace {

int launch_residual(const phikron_erk_s& E, const double* U, const double* S, double* D, cudaStream_t st) {
  launch_begin(KC_OTHER, st);
  residual_kernel<<<ew_blocks(E.N), EW, 0, st>>>(E.nonlin, U, E.Au, S, D, E.N);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

int launch_combine(const phikron_erk_s& E, const double* base, std::vector<std::pair<double, const double*>> terms,
                   double* out, cudaStream_t st) {
  Comb cb{};
  cb.nx = (int)terms.size();
  for (int k = 0; k < cb.nx; ++k) {
    cb.c[k] = terms[k].first;
    cb.X[k] = terms[k].second;
  }
  launch_begin(KC_OTHER, st);
  combine_kernel<<<ew_blocks(E.N), EW, 0, st>>>(base, cb, out, E.N);
  launch_end(st);
  PK_CHECK_LAUNCH();
  return PHIKRON_OK;
}

// one step of the method on U (in place)
int erk_step(phikron_erk_s& E, double* U, cudaStream_t st) {
  const long long N = E.N;
  const double tau = E.tau;
  launch_begin(KC_OTHER, st);
  kron_csr_kernel<<<ew_blocks(N), EW, 0, st>>>(E.K, U, E.Au, N);
  launch_end(st);
  PK_CHECK_LAUNCH();
  PK_RET(launch_residual(E, U, nullptr, E.D1, st));  // D1 = f(u) - Au
  if (E.method == PHIKRON_ERK_EULER) {
    PK_RET(phikron_apply(E.plans[0], E.D1, E.Out, st));
    return launch_combine(E, U, {{tau, E.Out + N}}, U, st);
  }
  const double c2 = E.cs[0];
  // U2 = u + tau c2 phi_1(-c2 tau A) D1
  PK_RET(phikron_apply(E.plans[0], E.D1, E.Out, st));
  PK_RET(launch_combine(E, U, {{tau * c2, E.Out + N}}, E.U2, st));
  PK_RET(launch_residual(E, E.U2, nullptr, E.D2, st));  // D2 = f(U2) - Au
  if (E.method == PHIKRON_ERK_RK2) {
    // u+ = u + tau phi_1(-tau A) ((1 - 1/(2c2)) D1 + 1/(2c2) D2)
    const double b2 = 1.0 / (2.0 * c2);
    PK_RET(launch_combine(E, nullptr, {{1.0 - b2, E.D1}, {b2, E.D2}}, E.V2, st));
    PK_RET(phikron_apply(E.plans[1], E.V2, E.Out, st));
    return launch_combine(E, U, {{tau, E.Out + N}}, U, st);
  }
  // RK3: the plan at c3 tau acts on [D1, D2 - D1] (outputs phi_0..phi_2 per rhs, 3N each)
  const double a = 4.0 / (9.0 * c2);
  PK_RET(launch_combine(E, E.D2, {{-1.0, E.D1}}, E.V2 + N, st));
  PK_TRY_CUDA(cudaMemcpyAsync(E.V2, E.D1, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  PK_RET(phikron_apply_many(E.plans[1], 2, E.V2, E.Out, st));
  // U3 = u + tau (2/3 phi_1,3 D1 + a phi_2,3 (D2 - D1))
  PK_RET(launch_combine(E, U, {{tau * 2.0 / 3.0, E.Out + N}, {tau * a, E.Out + 5 * N}}, E.U2, st));
  PK_RET(launch_residual(E, E.U2, E.D1, E.V2 + N, st));  // D3 - D1 = f(U3) - Au - D1
  PK_RET(phikron_apply_many(E.plans[2], 2, E.V2, E.Out, st));
  // u+ = u + tau (phi_1 D1 + 3/2 phi_2 (D3 - D1))
  return launch_combine(E, U, {{tau, E.Out + N}, {tau * 1.5, E.Out + 5 * N}}, U, st);
}

}  // namespace

extern "C" {

int phikron_erk_create(phikron_erk_t* out, int method, int dims, const double* const* A, const int* n, double tau,
                       double tol, int nonlinearity, const phikron_opts* opts) {
  clear_error();
  if (!out) { set_error("phikron_erk_create: out is NULL"); return PHIKRON_EINVAL; }
  *out = nullptr;
  if (method != PHIKRON_ERK_EULER && method != PHIKRON_ERK_RK2 && method != PHIKRON_ERK_RK3) {
    set_error("phikron_erk_create: method must be PHIKRON_ERK_EULER, _RK2 or _RK3");
    return PHIKRON_EINVAL;
  }
  if (nonlinearity != PHIKRON_NONLIN_NONE && nonlinearity != PHIKRON_NONLIN_ALLEN_CAHN) {
    set_error("phikron_erk_create: unknown nonlinearity");
    return PHIKRON_EINVAL;
  }
  if (!(tau > 0.0) || !std::isfinite(tau)) { set_error("phikron_erk_create: tau must be > 0"); return PHIKRON_EINVAL; }
  if (dims < 1 || dims > PHIKRON_MAX_DIMS || !A || !n) {
    set_error("phikron_erk_create: dims must be in 1..PHIKRON_MAX_DIMS");
    return PHIKRON_EINVAL;
  }
  phikron_opts o;
  phikron_opts_default(&o);
  if (opts) o = *opts;
  if (o.half_step) { set_error("phikron_erk_create: half_step is not used by the drivers"); return PHIKRON_EINVAL; }
  phikron_erk_s* E = alloc_fault() ? nullptr : new (std::nothrow) phikron_erk_s();
  if (!E) { set_error("phikron_erk_create: host allocation failed"); return PHIKRON_ENOMEM; }
  E->method = method;
  E->dims = dims;
  E->nonlin = nonlinearity;
  E->tau = tau;
  E->N = 1;
  for (int d = 0; d < dims; ++d) {
    if (!A[d] || n[d] < 1) {
      delete E;
      set_error("phikron_erk_create: bad factor");
      return PHIKRON_EINVAL;
    }
    E->n[d] = n[d];
    E->N *= n[d];
  }
  int rc = PHIKRON_OK;
  do {
    // plans: one per distinct c_j tau, phi_0 skipped
    if (method == PHIKRON_ERK_EULER) {
      E->cs = {1.0};
      E->lmax = {1};
    } else if (method == PHIKRON_ERK_RK2) {
      E->cs = {0.5, 1.0};
      E->lmax = {1, 1};
    } else {
      E->cs = {1.0 / 3.0, 2.0 / 3.0, 1.0};
      E->lmax = {1, 2, 2};
    }
    for (size_t k = 0; k < E->cs.size() && rc == PHIKRON_OK; ++k) {
      phikron_opts po = o;
      po.skip_phi0 = 1;
      po.max_rhs = (method == PHIKRON_ERK_RK3 && k > 0) ? 2 : 1;
      phikron_plan_t p = nullptr;
      rc = phikron_plan(&p, dims, A, n, E->cs[k] * tau, E->lmax[k], tol, &po);
      if (rc == PHIKRON_OK) E->plans.push_back(p);
    }
    if (rc != PHIKRON_OK) break;
    cudaGetDevice(&E->device);
    // CSR of every factor (nonzeros only)
    E->K.dims = dims;
    for (int d = 0; d < dims && rc == PHIKRON_OK; ++d) {
      const int nd = n[d];
      std::vector<int> rp(nd + 1, 0), cl;
      std::vector<double> vl;
      for (int i = 0; i < nd; ++i) {
        for (int j = 0; j < nd; ++j) {
          const double v = A[d][(size_t)i * nd + j];
          if (v != 0.0) {
            cl.push_back(j);
            vl.push_back(v);
          }
        }
        rp[i + 1] = (int)cl.size();
      }
      void *drp, *dcl, *dvl;
      if ((rc = E->alloc(&drp, sizeof(int) * rp.size())) != PHIKRON_OK) break;
      if ((rc = E->alloc(&dcl, sizeof(int) * std::max<size_t>(1, cl.size()))) != PHIKRON_OK) break;
      if ((rc = E->alloc(&dvl, sizeof(double) * std::max<size_t>(1, vl.size()))) != PHIKRON_OK) break;
      cudaMemcpy(drp, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice);
      if (!cl.empty()) {
        cudaMemcpy(dcl, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dvl, vl.data(), sizeof(double) * vl.size(), cudaMemcpyHostToDevice);
      }
      E->K.f[d] = Csr{(const int*)drp, (const int*)dcl, (const double*)dvl};
      E->K.n[d] = nd;
    }
    if (rc != PHIKRON_OK) break;
    const size_t vb = sizeof(double) * (size_t)E->N;
    if ((rc = E->alloc((void**)&E->Au, vb)) != PHIKRON_OK) break;
    if ((rc = E->alloc((void**)&E->D1, vb)) != PHIKRON_OK) break;
    if ((rc = E->alloc((void**)&E->D2, vb)) != PHIKRON_OK) break;
    if ((rc = E->alloc((void**)&E->U2, vb)) != PHIKRON_OK) break;
    if ((rc = E->alloc((void**)&E->V2, 2 * vb)) != PHIKRON_OK) break;
    if ((rc = E->alloc((void**)&E->Out, 6 * vb)) != PHIKRON_OK) break;
    if (cudaGetLastError() != cudaSuccess) { set_error("phikron_erk_create: CUDA error"); rc = PHIKRON_ECUDA; }
  } while (0);
  if (rc != PHIKRON_OK) {
    delete E;
    return rc;
  }
  *out = E;
  return PHIKRON_OK;
}

int phikron_erk_step(phikron_erk_t erk, double* U, int nsteps, void* stream) {
  clear_error();
  if (!erk || !U || nsteps < 0) { set_error("phikron_erk_step: bad argument"); return PHIKRON_EINVAL; }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) { set_error("cudaGetDevice failed"); return PHIKRON_ECUDA; }
  if (erk->device >= 0 && erk->device != prev) cudaSetDevice(erk->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = PHIKRON_OK;
  ProfScope ps(&erk->prof);
  const chk::Range r[1] = {{U, sizeof(double) * (size_t)erk->N}};
  chk::CallScope cs(st, r, 1);
  rc = cs.rc;
  for (int k = 0; k < nsteps && rc == PHIKRON_OK; ++k) rc = erk_step(*erk, U, st);
  if (erk->device >= 0 && erk->device != prev) cudaSetDevice(prev);
  return rc;
}

int phikron_erk_get_info(phikron_erk_t erk, phikron_erk_info* info) {
  clear_error();
  if (!erk || !info) { set_error("phikron_erk_get_info: NULL argument"); return PHIKRON_EINVAL; }
  *info = phikron_erk_info{};
  info->method = erk->method;
  info->nplans = (int)erk->plans.size();
  info->applies_per_step = (erk->method == PHIKRON_ERK_EULER) ? 1 : (erk->method == PHIKRON_ERK_RK2 ? 2 : 5);
  for (size_t k = 0; k < erk->plans.size(); ++k) {
    phikron_info pi;
    int rc = phikron_plan_info(erk->plans[k], &pi);
    if (rc != PHIKRON_OK) return rc;
    info->c[k] = erk->cs[k];
    info->s[k] = pi.s;
    info->m[k] = pi.m;
    info->actions[k] = pi.actions;
  }
  return PHIKRON_OK;
}

int phikron_erk_check_status(phikron_erk_t erk) {
  clear_error();
  if (!erk) { set_error("phikron_erk_check_status: NULL argument"); return PHIKRON_EINVAL; }
  for (phikron_plan_t p : erk->plans) {
    const int rc = phikron_check_status(p);
    if (rc != PHIKRON_OK) return rc;
  }
  return PHIKRON_OK;
}

int phikron_erk_profile_begin(phikron_erk_t erk, int max_timed) {
  clear_error();
  if (!erk || max_timed < 0) { set_error("phikron_erk_profile_begin: bad arguments"); return PHIKRON_EINVAL; }
  for (phikron_plan_t p : erk->plans) PK_RET(phikron_profile_begin(p, max_timed));
  return profiler_begin(erk->prof, max_timed);
}

int phikron_erk_profile_end(phikron_erk_t erk, phikron_profile* out) {
  clear_error();
  if (!erk || !out) { set_error("phikron_erk_profile_end: NULL argument"); return PHIKRON_EINVAL; }
  phikron_profile sum{};
  for (phikron_plan_t p : erk->plans) {
    phikron_profile one{};
    PK_RET(phikron_profile_end(p, &one));
    for (int c = 0; c < PHIKRON_KERNEL_CLASSES; ++c) {
      sum.ms[c] += one.ms[c];
      sum.launches[c] += one.launches[c];
    }
    sum.timed_launches += one.timed_launches;
  }
  PK_RET(profiler_end(erk->prof, &sum));
  *out = sum;
  return PHIKRON_OK;
}

void phikron_erk_destroy(phikron_erk_t erk) { delete erk; }

}  // extern "C"

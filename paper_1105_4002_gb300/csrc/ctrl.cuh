// Scalar control of GP, GPBB (Alg. 1), BT (Alg. 2) and UPN (Alg. 3).
//
// Runs in one thread (thread 0 of the block that finishes a reducing kernel),
// in FP64, on the device-resident DevState.  No thread ever waits here.
// A solver pass is two kernels: the back projection (gradient at the newly
// accepted point, then ctrl_after_grad) and the trial kernel (projected step,
// forward projection, in UPN the extrapolation for the case of acceptance,
// then ctrl_trial, or ctrl_trial2 for GPBB's two trial points).
//
// The acceptance tests are evaluated in Bregman form.  For f = phi and a step
// d = xbar - p from a base point p with gradient g = grad f(p),
//     f(xbar) - f(p) - g^T d = 1/2 ||A d||^2 + alpha * sum_j B_h(D_j xbar; D_j p),
// exactly (the data term is quadratic; B_h is the Bregman divergence of the
// Huber function).  The kernels deliver ||A d||^2 (A d gathered directly,
// not as a difference of two residuals), g^T d and sum_j B_h, each accurate
// relative to its own size, so the tests keep their meaning at step sizes
// where f(xbar) and f(p) agree to all float32 digits.  The tests themselves
// are the paper's, rearranged:
//   BT  (Alg. 2)  reject iff  B > L/2 ||d||^2          [f(x) > f(y) + g^T d + L/2 ||d||^2]
//   GPBB (Alg. 1) reject iff  (f_k - fhat) + (1 - sigma) g^T d + B >= 0
//                                                     [f(xbar) >= fhat - sigma g^T (x - xbar)]
//   mu-estimate   M(x, y) = B(x; y) / (1/2 ||x - y||^2)     (eq. mu_k_estimate)
// GPBB keeps f(x^(k)) as f(x^(0)) plus the exact increments g^T d + B.
#pragma once

#include "tvr_internal.cuh"

__device__ __forceinline__ void st_finish(DevState *st, int status) {
  st->done = 1;
  st->status = status;
}

__device__ __forceinline__ void st_hist(DevState *st, double a, double b, double c, double d,
                                        double e, double f, double g, double h) {
  if (st->hist && st->hist_used < st->hist_cap) {
    double *r = st->hist + (int64_t)st->hist_used * TVR_HIST_FIELDS;
    r[0] = a; r[1] = b; r[2] = c; r[3] = d; r[4] = e; r[5] = f; r[6] = g; r[7] = h;
    st->hist_used++;
  }
}

// Gradient-map stopping rule (Sec. III-D) after an accepted iteration.
__device__ __forceinline__ void st_stop_test(DevState *st) {
  double v;
  if (st->stop_mode == TVR_STOP_PER_N)
    v = st->gnorm / (double)st->N;
  else
    v = st->gnorm0 > 0.0 ? st->gnorm / st->gnorm0 : 0.0;
  st->stopval = v;
  if (!isfinite(st->gnorm)) {
    st_finish(st, TVR_ERR_NONFINITE);
    return;
  }
  if (v <= st->eps) {
    st_finish(st, TVR_OK);
    return;
  }
  if (st->k >= st->kmax) st_finish(st, TVR_NOT_CONVERGED);
}

template <typename T>
__device__ __forceinline__ void st_swap(T *&a, T *&b) {
  T *t = a;
  a = b;
  b = t;
}

// After the initial phi and gradient at x^(0): tot[0] = TV_tau(x^(0)).
__device__ __forceinline__ void ctrl_init(DevState *st, const double *tot) {
  st->f_evals = 1;
  st->g_evals = 1;
  st->f_cur = 0.5 * st->r_init[0] + st->alpha * tot[0];
  st->k = 0;
  st->trial = 0;
  st->need_grad = 0;
  st->done = 0;
  st->status = TVR_NOT_CONVERGED;
  st->total_trials = 0;
  st->hist_used = 0;
  st->gnorm = st->gnorm0 = st->stopval = 0.0;
  if (!isfinite(st->f_cur)) {
    st_finish(st, TVR_ERR_NONFINITE);
    return;
  }
  switch (st->solver) {
    case SOLVER_GPBB:
      st->theta = 1.0;  // theta_0 = 1
      st->beta = st->beta0;
      st->step = st->beta * st->theta;
      st->step2 = st->theta;
      st->fhist[0] = st->f_cur;
      st->nhist = 1;
      break;
    case SOLVER_UPN:
      st->mu = st->mubar;
      st->beta = 0.0;
      st->beta_prev = 0.0;
      st->M_valid = 0;
      st->Lt = st->Lbar;
      st->L = st->Lbar;
      st->step = 1.0 / st->Lt;
      break;
    default:  // GP
      st->Lt = st->Lbar;
      st->L = st->Lbar;
      st->step = 1.0 / st->Lt;
      break;
  }
}

// After a gradient evaluation at the newly accepted point.
// GPBB: tot[1] = <s, g_new - g_old>, tot[2] = ||s||^2, s = x^(k) - x^(k-1).
// UPN:  tot[1] = sum_j B_h(D_j x^(k); D_j y^(k)) (formed by the accepted trial).
__device__ __forceinline__ void ctrl_after_grad(DevState *st, const double *tot) {
  st->g_evals++;
  st->need_grad = 0;
  st->trial = 0;
  if (st->solver == SOLVER_GPBB) {
    st_swap(st->vN[RN_G], st->vN[RN_GN]);
    const double sy = tot[1], ss = tot[2];
    if (sy > 0.0 && ss > 0.0 && isfinite(sy) && isfinite(ss)) st->theta = ss / sy;  // BB step
    st->beta = st->beta0;
    st->step = st->beta * st->theta;
    st->step2 = st->theta;
  } else if (st->solver == SOLVER_UPN) {
    // M(x^(k), y^(k)) with x - y = -beta (x^(k) - x^(k-1)), A(x - y) = -beta u
    const double b2 = st->beta * st->beta;
    const double den = 0.5 * b2 * st->r_yf[0];
    const double num = 0.5 * b2 * st->r_yf[1] + st->alpha * tot[1];
    st->M_valid = 0;
    if (den > 1e-300) {
      const double M = num / den;
      if (isfinite(M)) {
        st->M = M;
        st->M_valid = 1;
      }
    }
    st->step = 1.0 / st->Lt;
  } else {
    st->step = 1.0 / st->Lt;
  }
}

// UPN (Alg. 3) scalars that acceptance at L would give: mu_k (eq.
// mu_k_estimate, kept non-increasing), theta_{k+1} (positive root of
// theta^2 = (1 - theta) theta_k^2 + (mu_k / L_k) theta) and beta_k.  Used by
// ctrl_trial and, speculatively, by the trial kernel.
__device__ __forceinline__ double upn_next(const DevState *st, double L, double &theta_new,
                                           double &mu_new) {
  if (st->k == 0) {
    mu_new = st->mubar;
    const double q = mu_new / L;
    theta_new = sqrt(q < 1.0 ? q : 1.0);
    return 0.0;  // y^(1) = x^(1)
  }
  mu_new = st->mu;
  if (st->M_valid) {
    const double M = st->M > 0.0 ? st->M : 0.0;
    mu_new = M < mu_new ? M : mu_new;
  }
  const double th = st->theta, q = mu_new / L;
  const double a = th * th - q;
  theta_new = 0.5 * (-a + sqrt(a * a + 4.0 * th * th));
  return th * (1.0 - th) / (th * th + theta_new);
}

// Accept / reject the trial point.  r_step = {g^T d, ||d||^2, sum B_h, GPBB ||x - P(x - theta g)||^2};
// fwd = {||A xbar - b||^2, ||A d||^2}.
__device__ __forceinline__ void ctrl_trial(DevState *st, const double *fwd) {
  st->f_evals++;
  const double gd = st->r_step[0], dd = st->r_step[1], btv = st->r_step[2];
  const double B = 0.5 * fwd[1] + st->alpha * btv;
  if (!isfinite(B) || !isfinite(gd) || !isfinite(dd)) {
    st_finish(st, TVR_ERR_NONFINITE);
    return;
  }
  if (st->solver == SOLVER_GPBB) {
    if (st->trial == 0) st->gnorm_trial = sqrt(st->r_step[3]) / st->theta;  // nu = 1/theta_k
    const int K1 = st->K + 1;
    const int cnt = st->nhist < K1 ? st->nhist : K1;
    double fhat = -INFINITY;
    for (int i = 0; i < cnt; ++i) {
      const double fv = st->fhist[(st->nhist - 1 - i) % TVR_FHIST];
      fhat = fv > fhat ? fv : fhat;
    }
    const double lhs = (st->f_cur - fhat) + (1.0 - st->sigma) * gd + B;
    if (lhs >= 0.0) {
      st->trial++;
      st->total_trials++;
      if (st->trial > st->max_trials) {
        st_finish(st, TVR_ERR_LINESEARCH);
        return;
      }
      st->beta = st->beta * st->beta;
      st->step = st->beta * st->theta;
      return;
    }
    st->f_cur = st->f_cur + gd + B;
    st->fhist[st->nhist % TVR_FHIST] = st->f_cur;
    st->nhist++;
    st->gnorm = st->gnorm_trial;
    if (st->k == 0) st->gnorm0 = st->gnorm;
    st_swap(st->vN[RN_X], st->vN[RN_T]);
    st_swap(st->vM[RM_R], st->vM[RM_RT]);
    st_swap(st->vM[RM_RS], st->vM[RM_RTS]);
    st_swap(st->w, st->wt);
    const int tr = st->trial;
    st->trial = 0;
    st->need_grad = 1;
    st->k++;
    st_stop_test(st);
    st_hist(st, st->k - 1, st->gnorm, st->theta, 0.0, st->beta, tr, st->f_cur, st->stopval);
    return;
  }
  // BT (GP and UPN)
  if (B > 0.5 * st->Lt * dd) {
    st->trial++;
    st->total_trials++;
    if (st->trial > st->bt_max) {
      st_finish(st, TVR_ERR_LINESEARCH);
      return;
    }
    st->Lt = st->rho * st->Lt;
    st->step = 1.0 / st->Lt;
    return;
  }
  st->L = st->Lt;
  st->f_cur = 0.5 * fwd[0] + st->alpha * st->r_step[4];  // phi(x+) of the accepted trial
  st->gnorm = st->L * sqrt(dd);  // ||G_{L_k}(base)|| = L_k ||base - x+||
  if (st->k == 0) st->gnorm0 = st->gnorm;
  if (st->solver == SOLVER_UPN) {
    double tn, mun;
    const double bnew = upn_next(st, st->L, tn, mun);
    st->mu = mun;
    st->theta = tn;
    st->beta_prev = st->beta;
    st->beta = bnew;
    if (st->spec_upn) {
      // adopt the extrapolation the trial formed for this outcome
      st_swap(st->vN[RN_Y], st->vN[RN_Y2]);
      st_swap(st->vM[RM_U], st->vM[RM_U2]);
      st_swap(st->vM[RM_RY], st->vM[RM_RY2]);
      st_swap(st->vM[RM_RYS], st->vM[RM_RYS2]);
      for (int i = 0; i < 3; ++i) st->r_yf[i] = st->r_spec[i];
    }
  }
  st_swap(st->vN[RN_X], st->vN[RN_T]);
  st_swap(st->vM[RM_R], st->vM[RM_RT]);
  st_swap(st->vM[RM_RS], st->vM[RM_RTS]);
  if (st->solver != SOLVER_UPN || st->spec_upn) st_swap(st->w, st->wt);
  const int tr = st->trial;
  st->trial = 0;
  st->need_grad = 1;
  st->k++;
  st->step = 1.0 / st->Lt;
  st_stop_test(st);
  st_hist(st, st->k - 1, st->gnorm, st->L, st->solver == SOLVER_UPN ? st->mu : 0.0,
          st->solver == SOLVER_UPN ? st->beta : 0.0, tr, st->f_cur, st->stopval);
}

// GPBB with two trial points per pass: fwd = {||A xbar - b||^2, ||A d||^2} of
// the first point (its step sums in r_step); the second point, at the step
// beta^2 theta that a rejection of the first leads to, has its sums in
// r_fwd2 / r_step2 and its vectors in the roles T2, RT2, RTS2, wt2.  The
// first is tested as usual; if it is rejected (and the trial cap not hit),
// the roles of the second point move into place and it is tested as the next
// trial, so the decisions and iterates are those of one point per pass.
__device__ __forceinline__ void ctrl_trial2(DevState *st, const double *fwd) {
  const int k0 = st->k;
  ctrl_trial(st, fwd);
  if (st->done || st->k != k0) return;  // accepted, or stopped
  st_swap(st->vN[RN_T], st->vN[RN_T2]);
  st_swap(st->vM[RM_RT], st->vM[RM_RT2]);
  st_swap(st->vM[RM_RTS], st->vM[RM_RTS2]);
  st_swap(st->wt, st->wt2);
  st->r_fwd[0] = st->r_fwd2[0];
  st->r_fwd[1] = st->r_fwd2[1];
  st->r_step[0] = st->r_step2[0];
  st->r_step[1] = st->r_step2[1];
  st->r_step[2] = st->r_step2[2];
  st->r_step[4] = st->r_step2[3];
  ctrl_trial(st, st->r_fwd2);
}

// Plain float64 lower-level solve: one kernel per step of Alg. 2 with every
// intermediate in HBM.  It computes the same iteration as the fused kernel
// (Step 1 by Eq. over_3, Eqs. split_xy .. update_lagrange, then the scoring of
// Alg. 1 line 9), in float64, and serves as the GPU reference path.
//
// Kernels per solve: step1, then for it = 0..K-1 {forward, project, transpose,
// update}, then forward and score.  Sample j belongs to scene sample_scene[j].
#include "internal.cuh"

namespace plan {
namespace {

__device__ __forceinline__ int scene_of(const int* sample_scene, int j) { return sample_scene[j]; }

// Step 1 (xi_bar = Gs p_axis + Hs b_axis), xi^0 = xi_bar, lambda^0 = 0 and the
// constant part M xi_bar + C b of the xi-step.  b_axis: the initial state and,
// with goal entries, x_f (x axis) or y_f and ydot_f = 0 (y axis), per sample.
// One 32-thread block per sample, thread = coefficient slot (axis = slot / 16,
// k = slot % 16).
__global__ void step1_kernel(const DevScene* scenes, const int* sample_scene, const double* p,
                             Consts c, Params prm, Plain64Work w) {
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  const int n = prm.n, ns = prm.n_seg, ne = c.ne;
  const int axis = lane >> 4, k = lane & 15;
  const bool valid = k < n;
  const DevScene& sc = scenes[scene_of(sample_scene, j)];
  const double* pj = p + size_t(j) * prm.d_p;
  __shared__ double xb[32];
  double b[5] = {sc.ego[axis], sc.ego[axis + 2], sc.ego[axis + 4], 0.0, 0.0};
  if (prm.goal) b[3] = pj[2 * ns + axis];
  if (valid) {
    const double* s1 = c.s1_64 + size_t(axis * n + k) * (ns + ne);
    double v = 0.0;
    for (int q = 0; q < ns; ++q) v += s1[q] * pj[(axis == 0 ? ns : 0) + q];
    for (int e = 0; e < ne; ++e) v += s1[ns + e] * b[e];
    xb[lane] = v;
    w.xi[size_t(j) * 32 + lane] = v;
    w.lam[size_t(j) * 32 + lane] = 0.0;
  }
  __syncthreads();
  if (valid) {
    const double* row = c.pj64 + size_t((sc.n_obs * 2 + axis) * n + k) * (2 * n + ne);
    double v = 0.0;
    for (int e = 0; e < ne; ++e) v += row[2 * n + e] * b[e];
    for (int i = 0; i < n; ++i) v += row[i] * xb[axis * 16 + i];
    w.xibarp[size_t(j) * 32 + lane] = v;
  }
}

// x, y, xd, yd, xdd, ydd at (sample, t) through Eq. (param).
__global__ void forward_kernel(int total, Consts c, Params prm, Plain64Work w) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = prm.m, n = prm.n;
  if (idx >= total * m) return;
  const int j = idx / m, t = idx % m;
  const double* xi = w.xi + size_t(j) * 32;
  double o[6] = {0, 0, 0, 0, 0, 0};
  for (int mat = 0; mat < 3; ++mat) {
    const double* row = c.basis64 + size_t(mat) * m * n + size_t(t) * n;
    double ax = 0.0, ay = 0.0;
    for (int k = 0; k < n; ++k) {
      ax += row[k] * xi[k];
      ay += row[k] * xi[16 + k];
    }
    o[2 * mat] = ax;
    o[2 * mat + 1] = ay;
  }
  double* st = w.state + size_t(j) * 6 * m;
  for (int q = 0; q < 6; ++q) st[q * m + t] = o[q];
}

// Eq. split_alpha_o with the clips of Eqs. clip_d_o, clip_d_v, clip_d_a and the
// slack of Eq. update_slack, stored as the residual rows h - F xi and
// e - s - G xi (per t: obstacle sum x, y; velocity x, y; acceleration x, y; lane).
// Closed forms without trigonometry: with (dx, dy) = p - o and the scaled
// distance d of an obstacle, cos(alpha) = dx / (a d) and sin(alpha) = dy / (b d),
// so the clipped point differs from p by (dx, dy)(1/d - 1) when d < 1 (at d = 0,
// atan2(0, 0) = 0 gives (a, 0)) and by zero otherwise.  The test d < 1 is
// dx^2 b^2 + dy^2 a^2 < a^2 b^2, free of divisions; only points inside an
// ellipse take the divisions and the reciprocal square root.  Velocity and
// acceleration directions come from one reciprocal square root of |v|^2, |a|^2.
// float64 division and square root are long instruction sequences on this part.
__global__ void project_kernel(int total, const DevScene* scenes, const int* sample_scene,
                               const double* obs, Params prm, Plain64Work w, int first) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = prm.m;
  if (idx >= total * m) return;
  const int j = idx / m, t = idx % m;
  const DevScene& sc = scenes[scene_of(sample_scene, j)];
  const double* st = w.state + size_t(j) * 6 * m;
  const double x = st[t], y = st[m + t], vx = st[2 * m + t], vy = st[3 * m + t];
  const double ax = st[4 * m + t], ay = st[5 * m + t];
  const double tt = t * prm.dt;

  double ex = 0.0, ey = 0.0;
  for (int i = 0; i < sc.n_obs; ++i) {
    const double* o = obs + size_t(sc.obs_off + i) * 6;
    const double dx = x - (o[0] + o[2] * tt), dy = y - (o[1] + o[3] * tt);
    const double a2 = o[4] * o[4], b2 = o[5] * o[5];
    if (fma(dx * dx, b2, dy * dy * a2) < a2 * b2) {      // d < 1
      const double sx = dx / o[4], sy = dy / o[5];
      const double d2 = fma(sx, sx, sy * sy);
      if (d2 > 0.0) {
        const double g = rsqrt(d2) - 1.0;
        ex += dx * g;
        ey += dy * g;
      } else {
        ex += o[4];
      }
    }
  }
  const double v2 = vx * vx + vy * vy;
  double sp = 0.0, cv = 1.0, sv = 0.0;
  if (v2 > 0.0) {
    const double rv = rsqrt(v2);
    sp = v2 * rv; cv = vx * rv; sv = vy * rv;
  }
  const double a2n = ax * ax + ay * ay;
  double am = 0.0, ca = 1.0, sa = 0.0;
  if (a2n > 0.0) {
    const double ra = rsqrt(a2n);
    am = a2n * ra; ca = ax * ra; sa = ay * ra;
  }
  const double S = fabs(sa * cv - ca * sv);
  double* da = w.da + size_t(j) * m;
  const double dap = first ? fmin(am, prm.a_max) : da[t];
  const double vmin_b = fmax(prm.v_min, sqrt(dap * S / prm.kappa_max));
  double vmax_b = prm.v_max;
  // road curvature at the previous iterate (Eq. clip_d_v), lane limits at this one
  double* xp = w.xprev + size_t(j) * m;
  const double xk = first ? x : xp[t];
  xp[t] = x;
  double kroad, ylb, yub, unused0, unused1;
  road_eval(sc, xk, &kroad, &unused0, &unused1);
  road_eval(sc, x, &unused0, &ylb, &yub);
  const double kr = fabs(kroad);
  if (kr * cv * cv > 0.0) vmax_b = fmin(prm.v_max, sqrt(prm.c_max / (kr * cv * cv)));
  const double dv = fmin(fmax(sp, vmin_b), vmax_b);
  const double kd = dv * dv * prm.kappa_max;
  const double amax_b = (S * prm.a_max <= kd) ? prm.a_max : kd / S;
  const double dan = fmin(fmax(am, 0.0), amax_b);
  da[t] = dan;
  const double s1 = fmax(0.0, yub - y), s2 = fmax(0.0, y - ylb);
  double* e = w.eps + size_t(j) * 7 * m;
  e[t] = ex;
  e[m + t] = ey;
  e[2 * m + t] = dv * cv - vx;
  e[3 * m + t] = dv * sv - vy;
  e[4 * m + t] = dan * ca - ax;
  e[5 * m + t] = dan * sa - ay;
  // G^T (e - s - G xi) per t: (y_ub - s1 - y) - (-y_lb - s2 + y)
  e[6 * m + t] = (yub - s1 - y) - (-ylb - s2 + y);
}

// w = F^T (h - F xi) + G^T (e - s - G xi): one 128-thread block per sample;
// warp q sums the timesteps t = q (mod 4) for every coefficient slot (lane),
// and the four partial sums are added in a fixed order.
constexpr int kTrWarps = 4;
__global__ void __launch_bounds__(32 * kTrWarps) transpose_kernel(Consts c, Params prm,
                                                                  Plain64Work w) {
  const int j = blockIdx.x, lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int m = prm.m, n = prm.n;
  const int axis = lane >> 4, k = lane & 15;
  __shared__ double part[kTrWarps][32];
  const double* e = w.eps + size_t(j) * 7 * m;
  const double* W0 = c.basis64;
  const double* W1 = c.basis64 + m * n;
  const double* W2 = c.basis64 + 2 * m * n;
  // two independent chains per warp (t = q + 8 i and t = q + 4 + 8 i)
  double acc[2] = {0.0, 0.0};
  if (k < n) {
    for (int t0 = q; t0 < m; t0 += 2 * kTrWarps) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int t = t0 + u * kTrWarps;
        if (t < m) {
          double e0 = e[axis * m + t];
          if (axis == 1) e0 += e[6 * m + t];
          acc[u] = fma(W0[t * n + k], e0, acc[u]);
          acc[u] = fma(W1[t * n + k], e[(2 + axis) * m + t], acc[u]);
          acc[u] = fma(W2[t * n + k], e[(4 + axis) * m + t], acc[u]);
        }
      }
    }
  }
  part[q][lane] = acc[0] + acc[1];
  __syncthreads();
  if (q == 0 && k < n)
    w.w[size_t(j) * 32 + lane] = (part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane]);
}

// lambda^it = lambda^{it-1} + rho/2 w (it > 0) and the xi-step.
__global__ void update_kernel(const DevScene* scenes, const int* sample_scene, Consts c,
                              Params prm, Plain64Work w, int it) {
  const int j = blockIdx.x, lane = threadIdx.x;
  const int n = prm.n;
  const int axis = lane >> 4, k = lane & 15;
  const bool valid = k < n;
  __shared__ double v[32], xo[32];
  const DevScene& sc = scenes[scene_of(sample_scene, j)];
  if (valid) {
    const size_t o = size_t(j) * 32 + lane;
    double lam = w.lam[o];
    const double wl = w.w[o];
    if (it > 0) lam += 0.5 * prm.rho * wl;
    w.lam[o] = lam;
    v[lane] = lam + prm.rho * wl;
    xo[lane] = w.xi[o];
  }
  __syncthreads();
  if (valid) {
    const double* row = c.pj64 + size_t((sc.n_obs * 2 + axis) * n + k) * (2 * n + c.ne);
    double acc = w.xibarp[size_t(j) * 32 + lane];
    for (int i = 0; i < n; ++i) acc += row[i] * v[axis * 16 + i] + row[n + i] * xo[axis * 16 + i];
    w.xi[size_t(j) * 32 + lane] = acc;
  }
}

// r_j and c_u of xi^K (one warp per sample, lanes over t), the xi output and
// the per-sample status (solution, residual and cost finite).
__global__ void score_kernel(const DevScene* scenes, const int* sample_scene, const double* obs,
                             Params prm, Plain64Work w, double* xi_out, double* r_out,
                             double* cu_out, int* st_out) {
  const int j = blockIdx.x, lane = threadIdx.x;
  const int m = prm.m, n = prm.n;
  const DevScene& sc = scenes[scene_of(sample_scene, j)];
  const double* st = w.state + size_t(j) * 6 * m;
  double r = 0.0, cu = 0.0;
  for (int t = lane; t < m; t += 32) {
    const double x = st[t], y = st[m + t], vx = st[2 * m + t], vy = st[3 * m + t];
    const double ax = st[4 * m + t], ay = st[5 * m + t];
    double kroad, ylb, yub;
    road_eval(sc, x, &kroad, &ylb, &yub);
    const double kr = fabs(kroad);
    const double tt = t * prm.dt;
    double coll = 0.0;
    for (int i = 0; i < sc.n_obs; ++i) {
      const double* o = obs + size_t(sc.obs_off + i) * 6;
      const double sx = (x - (o[0] + o[2] * tt)) / o[4], sy = (y - (o[1] + o[3] * tt)) / o[5];
      coll += fmax(0.0, 1.0 - sx * sx - sy * sy);
    }
    const double sp = sqrt(vx * vx + vy * vy);
    const double am = sqrt(ax * ax + ay * ay);
    const double kap = sp > 0.0 ? (ay * vx - ax * vy) / (sp * sp * sp) : 0.0;
    r += coll + fmax(0.0, sp - prm.v_max) + fmax(0.0, am - prm.a_max) +
         fmax(0.0, fabs(kap) - prm.kappa_max) + fmax(0.0, vx * vx * kr - prm.c_max) +
         fmax(0.0, y - yub) + fmax(0.0, ylb - y);
    cu += (sp - prm.v_max) * (sp - prm.v_max);
  }
  for (int o = 16; o >= 1; o >>= 1) {
    r += __shfl_xor_sync(0xffffffffu, r, o);
    cu += __shfl_xor_sync(0xffffffffu, cu, o);
  }
  if (lane == 0) { r_out[j] = r; cu_out[j] = cu; }
  const int axis = lane >> 4, k = lane & 15;
  const double xv = k < n ? w.xi[size_t(j) * 32 + lane] : 0.0;
  if (xi_out != nullptr && k < n) xi_out[size_t(j) * 2 * n + axis * n + k] = xv;
  if (st_out != nullptr) {
    const bool bad = __any_sync(0xffffffffu, !isfinite(xv)) || !isfinite(r) || !isfinite(cu);
    if (lane == 0) st_out[j] = bad ? PLAN_ENONFINITE : PLAN_OK;
  }
}

}  // namespace

cudaError_t launch_plain64(const DevScene* scenes, const Layout* layout, const int* sample_scene,
                           const double* obs, int total_B, const double* p, const Consts& c,
                           const Params& prm, const Plain64Work& w, double* xi_out, double* r,
                           double* cu, int* st, cudaStream_t s) {
  (void)layout;
  if (total_B == 0) return cudaSuccess;
  const int tm = total_B * prm.m;
  const int blk = 256, grid = (tm + blk - 1) / blk;
  step1_kernel<<<total_B, 32, 0, s>>>(scenes, sample_scene, p, c, prm, w);
  for (int it = 0; it < prm.K; ++it) {
    forward_kernel<<<grid, blk, 0, s>>>(total_B, c, prm, w);
    project_kernel<<<grid, blk, 0, s>>>(total_B, scenes, sample_scene, obs, prm, w, it == 0);
    transpose_kernel<<<total_B, 32 * kTrWarps, 0, s>>>(c, prm, w);
    update_kernel<<<total_B, 32, 0, s>>>(scenes, sample_scene, c, prm, w, it);
  }
  forward_kernel<<<grid, blk, 0, s>>>(total_B, c, prm, w);
  score_kernel<<<total_B, 32, 0, s>>>(scenes, sample_scene, obs, prm, w, xi_out, r, cu, st);
  return cudaGetLastError();
}

}  // namespace plan

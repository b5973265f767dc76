// The Step-1 QP of Alg. 1 line 7 as a differentiable layer (the learned
// sampler's optimization layer, Sec. IV: convex Step-1 cost and equality
// constraints, inequalities ignored).  Per axis the solution is affine in the
// set-points and the initial state:
//   xi_axis = Gs p_axis + Hs b_axis
// with the Step-1 map [Gs | Hs] formed from the float64 KKT inverse at
// context creation (rows of Consts::s1_64).  The backward pass is the
// transposed map: dL/dp_axis = Gs^T g_axis, dL/db_axis = Hs^T g_axis.
// x uses the velocity set-points p[n_seg..2 n_seg) and b = (x0, vx0, ax0); y
// the lateral offsets p[0..n_seg) and b = (y0, vy0, ay0).  Float64 throughout.
#include "internal.cuh"

namespace plan {
namespace {

// One thread per (sample, coefficient slot): xi[j][axis n + k].
__global__ void qp_forward_kernel(const double* __restrict__ s1, const double* __restrict__ p,
                                  const double* __restrict__ b0, int B, int n, int ns,
                                  double* __restrict__ xi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * 2 * n) return;
  const int j = e / (2 * n), r = e % (2 * n), axis = r / n;
  const double* row = s1 + size_t(r) * (ns + 3);
  const double* pj = p + size_t(j) * 2 * ns + (axis == 0 ? ns : 0);
  const double* bj = b0 + size_t(j) * 6;
  double v = 0.0;
  for (int q = 0; q < ns; ++q) v = fma(row[q], pj[q], v);
  v = fma(row[ns], bj[axis], v);
  v = fma(row[ns + 1], bj[axis + 2], v);
  v = fma(row[ns + 2], bj[axis + 4], v);
  xi[e] = v;
}

// One thread per (sample, input): dL/dp[j][a] for a < 2 n_seg, then
// dL/db0[j][i] for i < 6 (written only when grad_b0 is given).
__global__ void qp_backward_kernel(const double* __restrict__ s1, const double* __restrict__ g,
                                   int B, int n, int ns, double* __restrict__ grad_p,
                                   double* __restrict__ grad_b0) {
  const int per = 2 * ns + 6;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * per) return;
  const int j = e / per, a = e % per;
  int axis, col;
  if (a < 2 * ns) {
    axis = a < ns ? 1 : 0;             // p = [y_d (y axis) | v_d (x axis)]
    col = a < ns ? a : a - ns;
  } else {
    if (grad_b0 == nullptr) return;
    const int i = a - 2 * ns;          // b0 = (x, y, vx, vy, ax, ay)
    axis = i & 1;
    col = ns + i / 2;
  }
  const double* gj = g + size_t(j) * 2 * n + axis * n;
  double v = 0.0;
  for (int k = 0; k < n; ++k) v = fma(s1[size_t(axis * n + k) * (ns + 3) + col], gj[k], v);
  if (a < 2 * ns) grad_p[size_t(j) * 2 * ns + a] = v;
  else grad_b0[size_t(j) * 6 + (a - 2 * ns)] = v;
}

}  // namespace

cudaError_t launch_qp_forward(const Consts& c, const double* p, const double* b0, int B,
                              double* xi, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int total = B * 2 * c.n;
  qp_forward_kernel<<<(total + 255) / 256, 256, 0, s>>>(c.s1_64, p, b0, B, c.n, c.n_seg, xi);
  return cudaGetLastError();
}

cudaError_t launch_qp_backward(const Consts& c, const double* g, int B, double* grad_p,
                               double* grad_b0, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int total = B * (2 * c.n_seg + 6);
  qp_backward_kernel<<<(total + 255) / 256, 256, 0, s>>>(c.s1_64, g, B, c.n, c.n_seg, grad_p,
                                                          grad_b0);
  return cudaGetLastError();
}

}  // namespace plan

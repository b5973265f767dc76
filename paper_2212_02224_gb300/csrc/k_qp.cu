// The Step-1 QP of Alg. 1 line 7 as a differentiable layer (the learned
// sampler's optimization layer, Sec. IV: convex Step-1 cost and equality
// constraints, inequalities ignored).  Per axis the solution is affine in the
// set-points and the initial state:
//   xi_axis = Gs p_axis + Hs b_axis
// with the Step-1 map [Gs | Hs] formed from the float64 KKT inverse at
// context creation (rows of Consts::s1_64).  The backward pass is the
// transposed map: dL/dp_axis = Gs^T g_axis, dL/db_axis = Hs^T g_axis.
// x uses the velocity set-points p[n_seg..2 n_seg) and b = (x0, vx0, ax0); y
// the lateral offsets p[0..n_seg) and b = (y0, vy0, ay0).  With goal entries
// b also holds x_f = p[2 n_seg] (x) or y_f = p[2 n_seg + 1] and ydot_f = 0 (y),
// so their gradients are the transposed map's b columns.  Float64 throughout.
#include "internal.cuh"

namespace plan {
namespace {

// One thread per (sample, coefficient slot): xi[j][axis n + k].
__global__ void qp_forward_kernel(const double* __restrict__ s1, const double* __restrict__ p,
                                  const double* __restrict__ b0, int B, int n, int ns, int ne,
                                  int d_p, double* __restrict__ xi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * 2 * n) return;
  const int j = e / (2 * n), r = e % (2 * n), axis = r / n;
  const double* row = s1 + size_t(r) * (ns + ne);
  const double* pj = p + size_t(j) * d_p;
  const double* bj = b0 + size_t(j) * 6;
  double v = 0.0;
  for (int q = 0; q < ns; ++q) v = fma(row[q], pj[(axis == 0 ? ns : 0) + q], v);
  v = fma(row[ns], bj[axis], v);
  v = fma(row[ns + 1], bj[axis + 2], v);
  v = fma(row[ns + 2], bj[axis + 4], v);
  if (d_p > 2 * ns) v = fma(row[ns + 3], pj[2 * ns + axis], v);   // x_f or y_f
  xi[e] = v;
}

// One thread per (sample, input): dL/dp[j][a] for a < d_p, then dL/db0[j][i]
// for i < 6 (written only when grad_b0 is given).
__global__ void qp_backward_kernel(const double* __restrict__ s1, const double* __restrict__ g,
                                   int B, int n, int ns, int ne, int d_p,
                                   double* __restrict__ grad_p, double* __restrict__ grad_b0) {
  const int per = d_p + 6;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * per) return;
  const int j = e / per, a = e % per;
  int axis, col;
  if (a < 2 * ns) {
    axis = a < ns ? 1 : 0;             // p = [y_d (y axis) | v_d (x axis) | x_f, y_f]
    col = a < ns ? a : a - ns;
  } else if (a < d_p) {
    axis = a - 2 * ns;                 // x_f: x axis, y_f: y axis; column of the b entry
    col = ns + 3;
  } else {
    if (grad_b0 == nullptr) return;
    const int i = a - d_p;             // b0 = (x, y, vx, vy, ax, ay)
    axis = i & 1;
    col = ns + i / 2;
  }
  const double* gj = g + size_t(j) * 2 * n + axis * n;
  double v = 0.0;
  for (int k = 0; k < n; ++k) v = fma(s1[size_t(axis * n + k) * (ns + ne) + col], gj[k], v);
  if (a < d_p) grad_p[size_t(j) * d_p + a] = v;
  else grad_b0[size_t(j) * 6 + (a - d_p)] = v;
}

}  // namespace

cudaError_t launch_qp_forward(const Consts& c, const double* p, const double* b0, int B,
                              double* xi, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int total = B * 2 * c.n;
  const int d_p = 2 * c.n_seg + 2 * c.goal;
  qp_forward_kernel<<<(total + 255) / 256, 256, 0, s>>>(c.s1_64, p, b0, B, c.n, c.n_seg, c.ne,
                                                         d_p, xi);
  return cudaGetLastError();
}

cudaError_t launch_qp_backward(const Consts& c, const double* g, int B, double* grad_p,
                               double* grad_b0, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  const int d_p = 2 * c.n_seg + 2 * c.goal;
  const int total = B * (d_p + 6);
  qp_backward_kernel<<<(total + 255) / 256, 256, 0, s>>>(c.s1_64, g, B, c.n, c.n_seg, c.ne, d_p,
                                                          grad_p, grad_b0);
  return cudaGetLastError();
}

}  // namespace plan

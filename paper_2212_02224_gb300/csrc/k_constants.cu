// Per-configuration constants, formed and inverted in float64 on the GPU:
//   * the Bernstein basis W, Wd, Wdd of the trajectory parametrisation (Eq. param),
//   * the KKT inverse of the Step-1 QP (Alg. 1 line 7, Eq. over_2), folded into
//     the maps xi_bar = Gs p + Hs b per axis,
//   * the KKT inverse of the projection xi-step (Alg. 2, Eq. split_xy) for every
//     obstacle count N, folded into xi = M r + C b and MP = rho M P.
// The equality rows A of an axis (Eq. lower_eq) are the initial rows of
// Eq. boundary_cond_initial and, with goal entries in p, the final rows of
// Eq. final_boundary: x(t_f) = x_f; y(t_f) = y_f, ydot(t_f) = 0.
#include "internal.cuh"

namespace plan {
namespace {

__device__ double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// b_{k,deg}(tau), zero outside 0..deg
__device__ double bern(int deg, int k, double tau) {
  if (k < 0 || k > deg) return 0.0;
  double a = 1.0, b = 1.0;
  for (int i = 0; i < k; ++i) a *= tau;
  for (int i = 0; i < deg - k; ++i) b *= (1.0 - tau);
  return binom(deg, k) * a * b;
}

__global__ void basis_kernel(int m, int n, double dt, double* b64, float* b32) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  int t = idx / n, k = idx % n;
  int deg = n - 1;
  double tf = (m - 1) * dt;
  double tau = double(t) / double(m - 1);
  double w = bern(deg, k, tau);
  double wd = deg * (bern(deg - 1, k - 1, tau) - bern(deg - 1, k, tau)) / tf;
  double wdd = deg * (deg - 1) *
               (bern(deg - 2, k - 2, tau) - 2.0 * bern(deg - 2, k - 1, tau) + bern(deg - 2, k, tau)) /
               (tf * tf);
  b64[0 * m * n + t * n + k] = w;
  b64[1 * m * n + t * n + k] = wd;
  b64[2 * m * n + t * n + k] = wdd;
  const int st = basis32_stride(n), ncp = basis32_ncp(n);
  b32[t * st + 0 * ncp + k] = float(w);
  b32[t * st + 1 * ncp + k] = float(wd);
  b32[t * st + 2 * ncp + k] = float(wdd);
}

// Invert the (sz x sz) matrix held in smem `a` (leading dimension ld, with
// identity appended in columns sz..2sz-1) by Gauss-Jordan elimination with
// partial pivoting.  All threads of the block participate.
__device__ void gauss_jordan(double* a, int sz, int ld, int* piv_row) {
  for (int c = 0; c < sz; ++c) {
    if (threadIdx.x == 0) {
      int best = c;
      double bv = fabs(a[c * ld + c]);
      for (int r = c + 1; r < sz; ++r) {
        double v = fabs(a[r * ld + c]);
        if (v > bv) { bv = v; best = r; }
      }
      *piv_row = best;
    }
    __syncthreads();
    int pr = *piv_row;
    if (pr != c) {
      for (int j = threadIdx.x; j < 2 * sz; j += blockDim.x) {
        double t = a[c * ld + j];
        a[c * ld + j] = a[pr * ld + j];
        a[pr * ld + j] = t;
      }
    }
    __syncthreads();
    double inv = 1.0 / a[c * ld + c];
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * sz; j += blockDim.x) a[c * ld + j] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < sz * 2 * sz; e += blockDim.x) {
      int r = e / (2 * sz), j = e % (2 * sz);
      if (r == c) continue;
      double f = a[r * ld + c];
      // column c of row r is read by every j of that row: use the value read
      // before this phase (stored in column c, which is only zeroed below)
      if (j != c) a[r * ld + j] -= f * a[c * ld + j];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < sz; r += blockDim.x)
      if (r != c) a[r * ld + c] = 0.0;
    __syncthreads();
  }
}

// Entry i of equality row e of an axis: e = 0, 1, 2 are the rows of W, Wd,
// Wdd at t0; e = 3 the row of W at t_f; e = 4 the row of Wd at t_f.
__device__ double eq_entry(const Consts& c, int e, int i) {
  const int m = c.m, n = c.n;
  if (e < 3) return c.basis64[size_t(e) * m * n + i];
  return c.basis64[size_t(e - 3) * m * n + size_t(m - 1) * n + i];
}

// One block per job: job 0/1 = Step-1 x/y, job 2 + 2N + axis = projection.
__global__ void kkt_kernel(Consts c, Params p) {
  const int m = c.m, n = c.n, ns = c.n_seg;
  const int job = blockIdx.x;
  const double* W = c.basis64;
  const double* Wd = c.basis64 + m * n;
  const double* Wdd = c.basis64 + 2 * m * n;

  const bool step1 = job < 2;
  const int axis = step1 ? job : (job - 2) % 2;
  const int N = step1 ? 0 : (job - 2) / 2;
  const int ne = eq_rows(axis, c.goal);   // equality rows of this axis

  extern __shared__ double sh[];
  const int sz = n + ne, ld = 2 * sz;
  const int szmax = n + c.ne;
  double* a = sh;                      // sz x ld (room for szmax x 2 szmax)
  double* gram = a + szmax * 2 * szmax;   // n x n (P or Q/2 pieces)
  double* ext = gram + n * n;          // n x ns (L^T S) for step 1
  __shared__ int piv;

  // Gram matrix of the axis.
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e % n;
    double acc = 0.0;
    for (int t = 0; t < m; ++t) {
      double wi = W[t * n + i], wj = W[t * n + j];
      double di = Wd[t * n + i], dj = Wd[t * n + j];
      double ai = Wdd[t * n + i], aj = Wdd[t * n + j];
      if (step1) {
        // Q = 2 (Wdd^T Wdd + L^T L): c_s plus the tracking term of the axis
        double li, lj;
        if (axis == 0) { li = ai + p.kp_lon * di; lj = aj + p.kp_lon * dj; }
        else { li = ai + p.kv_lat * di + p.kp_lat * wi; lj = aj + p.kv_lat * dj + p.kp_lat * wj; }
        acc += 2.0 * (ai * aj + li * lj);
      } else {
        // P = N W^T W + Wd^T Wd + Wdd^T Wdd (+ G^T G = 2 W^T W on the y axis)
        double nw = double(N) + (axis == 1 ? 2.0 : 0.0);
        acc += nw * wi * wj + di * dj + ai * aj;
      }
    }
    gram[e] = acc;
  }
  if (step1) {
    // ext = L^T S: S[t][seg] = 1 when step t belongs to segment seg
    int q = m / ns, rem = m % ns;
    for (int e = threadIdx.x; e < n * ns; e += blockDim.x) {
      int i = e / ns, sg = e % ns;
      int t0 = sg * q + (sg < rem ? sg : rem);
      int len = q + (sg < rem ? 1 : 0);
      double acc = 0.0;
      for (int t = t0; t < t0 + len; ++t) {
        double li = (axis == 0) ? Wdd[t * n + i] + p.kp_lon * Wd[t * n + i]
                                : Wdd[t * n + i] + p.kv_lat * Wd[t * n + i] + p.kp_lat * W[t * n + i];
        acc += li;
      }
      ext[e] = acc;
    }
  }
  __syncthreads();
  // KKT matrix [[H, A^T], [A, 0]] with identity appended.
  for (int e = threadIdx.x; e < sz * ld; e += blockDim.x) {
    int r = e / ld, j = e % ld;
    double v = 0.0;
    if (j < sz) {
      if (r < n && j < n) {
        v = step1 ? gram[r * n + j] : p.rho * gram[r * n + j] + (r == j ? 1.0 : 0.0);
      } else if (r < n && j >= n) {
        v = eq_entry(c, j - n, r);        // A^T
      } else if (r >= n && j < n) {
        v = eq_entry(c, r - n, j);        // A
      }
    } else {
      v = (j - sz == r) ? 1.0 : 0.0;
    }
    a[e] = v;
  }
  __syncthreads();
  gauss_jordan(a, sz, ld, &piv);
  // inverse in columns sz..2sz-1
  const double* inv = a + sz;
  if (step1) {
    const double kp = axis == 0 ? p.kp_lon : p.kp_lat;
    const int stride = ns + c.ne;
    double* o64 = c.s1_64 + axis * n * stride;
    float* o32 = c.s1_32 + axis * n * stride;
    for (int e = threadIdx.x; e < n * stride; e += blockDim.x) {
      int k = e / stride, j = e % stride;
      double v;
      if (j < ns) {
        // xi_bar = Kinv11 (-q) with -q = 2 kp L^T S p_axis
        v = 0.0;
        for (int i = 0; i < n; ++i) v += inv[k * ld + i] * 2.0 * kp * ext[i * ns + j];
      } else {
        v = (j - ns < ne) ? inv[k * ld + n + (j - ns)] : 0.0;
      }
      o64[e] = v;
      o32[e] = float(v);
    }
  } else {
    const int stride = 2 * n + c.ne;
    double* o64 = c.pj64 + (N * 2 + axis) * n * stride;
    float* o32 = c.pj32 + (N * 2 + axis) * n * stride;
    for (int e = threadIdx.x; e < n * stride; e += blockDim.x) {
      int k = e / stride, j = e % stride;
      double v;
      if (j < n) {
        v = inv[k * ld + j];
      } else if (j < 2 * n) {
        int jj = j - n;
        v = 0.0;
        for (int i = 0; i < n; ++i) v += inv[k * ld + i] * gram[i * n + jj];
        v *= p.rho;
      } else {
        v = (j - 2 * n < ne) ? inv[k * ld + n + (j - 2 * n)] : 0.0;
      }
      o64[e] = v;
      o32[e] = float(v);
    }
  }
}

}  // namespace

cudaError_t build_constants(const Consts& c, const Params& p, cudaStream_t s) {
  int mn = c.m * c.n;
  cudaError_t e0 = cudaMemsetAsync(c.basis32, 0, sizeof(float) * c.m * basis32_stride(c.n), s);
  if (e0 != cudaSuccess) return e0;
  basis_kernel<<<(mn + 127) / 128, 128, 0, s>>>(c.m, c.n, p.dt, c.basis64, c.basis32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int sz = c.n + c.ne;
  size_t shm = sizeof(double) * (sz * 2 * sz + c.n * c.n + c.n * c.n_seg);
  int jobs = 2 + 2 * (c.max_obs + 1);
  kkt_kernel<<<jobs, 256, shm, s>>>(c, p);
  return cudaGetLastError();
}

}  // namespace plan

// Outer loop of Alg. 1 on the device: sampling (line 4), ConstraintEliteSet and
// EliteSet (lines 10-13), and the distribution update of Eqs. (mean_update,
// cov_update, s_formula), one thread block per scene, float64.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
// key = (seed_lo, seed_hi) and counter = (j, l | c << 16, step_lo, step_hi);
// Box-Muller turns word pairs (2q, 2q+1) into normals.
#include <atomic>

#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.cuh"

namespace plan {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double unit_open(unsigned w) { return (double(w) + 0.5) * 0x1p-32; }

// The Philox words of sample j in outer iteration l: entry e of p_j uses word
// e mod 4 of block e div 4.
__device__ __forceinline__ void philox_words(const DevCem& st, int j, int l, int d_p,
                                             unsigned (&w)[kMaxDp]) {
  const uint2 key = make_uint2(unsigned(st.seed & 0xffffffffull), unsigned(st.seed >> 32));
  for (int c = 0; c < (d_p + 3) / 4; ++c) {
    const uint4 ctr = make_uint4(unsigned(j), unsigned(l) | (unsigned(c) << 16),
                                 unsigned(st.step & 0xffffffffull), unsigned(st.step >> 32));
    const uint4 o = philox4x32_10(ctr, key);
    w[4 * c] = o.x;
    if (4 * c + 1 < kMaxDp) w[4 * c + 1] = o.y;
    if (4 * c + 2 < kMaxDp) w[4 * c + 2] = o.z;
    if (4 * c + 3 < kMaxDp) w[4 * c + 3] = o.w;
  }
}

// Standard normals z of sample j in outer iteration l (Box-Muller on the word
// pairs (2q, 2q+1)).  They depend only on the seed, the episode step, j and l,
// not on the distribution being sampled.
__device__ __forceinline__ void normals(const DevCem& st, int j, int l, int d_p,
                                        double (&z)[kMaxDp]) {
  unsigned w[kMaxDp];
  philox_words(st, j, l, d_p, w);
  for (int q = 0; 2 * q < d_p; ++q) {
    // Box-Muller: r (cos, sin)(2 pi u2); sincospi takes the angle as a
    // multiple of pi (2 u2 is exact), one argument reduction for both
    const double r = sqrt(-2.0 * log(unit_open(w[2 * q])));
    double sn, cs;
    sincospi(2.0 * unit_open(w[2 * q + 1]), &sn, &cs);
    z[2 * q] = r * cs;
    z[2 * q + 1] = r * sn;
  }
}

// Alg. 1 line 4 for every scene: grid (ceil(max_B / 128), S).  With zbuf the
// normals of the Gaussian draw were computed beforehand by normals_kernel
// (zbuf[(off + j) d_p + a]); without it they are computed here.
__global__ void sample_kernel(const DevScene* scenes, const Layout* layout, const DevCem* cem,
                              int l, Params prm, const double* zbuf, double* p) {
  pdl_wait();      // the distribution comes from the previous selection kernel
  pdl_trigger();
  const int s = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const Layout lay = layout[s];
  if (j >= lay.B) return;
  const DevCem& st = cem[s];
  const int d_p = prm.d_p, ns = prm.n_seg;
  double* out = p + size_t(lay.off + j) * d_p;
  if (l == 1 && st.fresh) {
    unsigned w[kMaxDp];
    philox_words(st, j, l, d_p, w);
    const DevScene& sc = scenes[s];
    for (int e = 0; e < ns; ++e) {
      int idx = int(floor(unit_open(w[e]) * sc.n_lanes));
      if (idx > sc.n_lanes - 1) idx = sc.n_lanes - 1;
      out[e] = (idx + 0.5) * sc.lane_width;
    }
    for (int e = ns; e < 2 * ns; ++e)
      out[e] = prm.v_des_lo + (prm.v_des_hi - prm.v_des_lo) * unit_open(w[e]);
    if (prm.goal) {
      // goal entries: x_f = x0 + v t_f with v ~ U[v_des_lo, v_des_hi], y_f a lane centre
      const double tf = (prm.m - 1) * prm.dt;
      const double v = prm.v_des_lo + (prm.v_des_hi - prm.v_des_lo) * unit_open(w[2 * ns]);
      out[2 * ns] = sc.ego[0] + tf * v;
      int idx = int(floor(unit_open(w[2 * ns + 1]) * sc.n_lanes));
      if (idx > sc.n_lanes - 1) idx = sc.n_lanes - 1;
      out[2 * ns + 1] = (idx + 0.5) * sc.lane_width;
    }
  } else {
    double z[kMaxDp];
    if (zbuf) {
      const double* zj = zbuf + size_t(lay.off + j) * d_p;
      for (int a = 0; a < d_p; ++a) z[a] = zj[a];
    } else {
      normals(st, j, l, d_p, z);
    }
    for (int a = 0; a < d_p; ++a) {
      double v = 0.0;
      for (int b = 0; b <= a; ++b) v = fma(z[b], st.chol[a * kMaxDp + b], v);
      out[a] = st.mu[a] + v;
    }
  }
}

// The normals of outer iteration l for every sample into zbuf: grid
// (ceil(max_B / 128), S).  It reads only the seed and the episode step, which
// no kernel of the cycle changes before the last selection, so it can run
// beside the solve of iteration l - 1.
__global__ void normals_kernel(const Layout* layout, const DevCem* cem, int l, Params prm,
                               double* zbuf) {
  const int s = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const Layout lay = layout[s];
  if (j >= lay.B) return;
  const int d_p = prm.d_p;
  double z[kMaxDp];
  normals(cem[s], j, l, d_p, z);
  double* out = zbuf + size_t(lay.off + j) * d_p;
  for (int a = 0; a < d_p; ++a) out[a] = z[a];
}

// Total order on doubles: -0 is +0, NaN sorts after everything.  Integer
// operations only (float64 compares would take the float64 pipe).
__device__ __forceinline__ unsigned long long ord_key(double v) {
  unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned long long mag = u & 0x7fffffffffffffffull;
  if (mag > 0x7ff0000000000000ull) return 0xfff8000000000000ull;   // canonical NaN, after +inf
  if (mag == 0ull) u = 0ull;                                        // -0 is +0
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

constexpr int kSelThreads = 1024;

struct SelShared {
  unsigned hist[256];
  unsigned wsum[32];
  unsigned long long key[kMaxEliteC];
  int idx[kMaxEliteC];
  double sw[kMaxEliteC];
  unsigned long long prefix;
  int need, digit, count;
  double acc[kMaxDp * kMaxDp + kMaxDp + 2];
};

// Block-wide exclusive prefix sum of one flag per thread; returns the prefix and
// writes the block total to *total.
__device__ int block_scan_flag(bool f, SelShared& sh, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  const int within = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) sh.wsum[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    unsigned v = sh.wsum[lane];
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    sh.wsum[lane] = incl - v;
    if (lane == 31) sh.count = int(incl);
  }
  __syncthreads();
  const int res = int(sh.wsum[warp]) + within;
  *total = sh.count;
  __syncthreads();
  return res;
}

// ConstraintEliteSet: indices of the n_c lowest r (ties to the lower index),
// written to sh.idx[0..n_c) in increasing index order.  Radix select on the
// 64-bit order key, then an ordered compaction.
__device__ void select_constraint_set(const double* r, int B, int n_c, SelShared& sh) {
  const int tid = threadIdx.x;
  if (tid == 0) { sh.prefix = 0ull; sh.need = n_c; }
  __syncthreads();
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) sh.hist[i] = 0u;
    __syncthreads();
    const unsigned long long pre = sh.prefix;
    for (int i = tid; i < B; i += blockDim.x) {
      const unsigned long long k = ord_key(r[i]);
      if (shift == 56 || ((k ^ pre) >> (shift + 8)) == 0ull)
        atomicAdd(&sh.hist[(k >> shift) & 255ull], 1u);
    }
    __syncthreads();
    if (tid < 32) {
      // lane handles digits [8 lane, 8 lane + 8)
      unsigned loc = 0;
      for (int d = 0; d < 8; ++d) loc += sh.hist[8 * tid + d];
      unsigned incl = loc;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += t;
      }
      const unsigned excl = incl - loc;
      const int need = sh.need;
      const unsigned hit = __ballot_sync(0xffffffffu, incl >= unsigned(need));
      const int first = __ffs(hit) - 1;
      if (tid == first) {
        unsigned cum = excl;
        int d = 8 * tid;
        for (; d < 8 * tid + 7; ++d) {
          if (cum + sh.hist[d] >= unsigned(need)) break;
          cum += sh.hist[d];
        }
        sh.need = need - int(cum);
        sh.prefix = pre | (static_cast<unsigned long long>(d) << shift);
      }
    }
    __syncthreads();
  }
  const unsigned long long T = sh.prefix;
  const int need_eq = sh.need;
  __syncthreads();
  for (int i = tid; i < n_c; i += blockDim.x) sh.idx[i] = -1;
  __syncthreads();
  int ties_before = 0, sel_before = 0;
  for (int base = 0; base < B; base += blockDim.x) {
    const int i = base + tid;
    bool less = false, eq = false;
    if (i < B) {
      const unsigned long long k = ord_key(r[i]);
      less = k < T;
      eq = k == T;
    }
    int tot_eq;
    const int eq_rank = block_scan_flag(eq, sh, &tot_eq) + ties_before;
    const bool sel = less || (eq && eq_rank < need_eq);
    int tot_sel;
    const int pos = block_scan_flag(sel, sh, &tot_sel) + sel_before;
    if (sel && pos < n_c) sh.idx[pos] = i;
    ties_before += tot_eq;
    sel_before += tot_sel;
  }
  __syncthreads();
}

// Sort sh.key / sh.idx [0, P) ascending by (key, idx), P a power of two.
__device__ void bitonic_sort(SelShared& sh, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool asc = (i & k) == 0;
          const unsigned long long ka = sh.key[i], kb = sh.key[ixj];
          const int ia = sh.idx[i], ib = sh.idx[ixj];
          const bool gt = (ka > kb) || (ka == kb && ia > ib);
          if (gt == asc) {
            sh.key[i] = kb; sh.key[ixj] = ka;
            sh.idx[i] = ib; sh.idx[ixj] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
}

// EliteSet: the q lowest (cu + r) among the n_c candidates in sh.idx, sorted
// ascending into sh.idx[0..q).
__device__ void select_elite_set(const double* r, const double* cu, int B, int n_c,
                                 SelShared& sh) {
  int P = 1;
  while (P < n_c) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int id = i < n_c ? sh.idx[i] : -1;
    if (id >= 0 && id < B) {
      sh.key[i] = ord_key(cu[id] + r[id]);
    } else {
      sh.key[i] = ~0ull;
      sh.idx[i] = 0x7fffffff;
    }
  }
  __syncthreads();
  bitonic_sort(sh, P);
}

// Sum over the warp in a fixed butterfly order (lane 0's result is used).
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Eqs. (mean_update, cov_update, s_formula) over the q elites p_e(e), costs c_e(e),
// with the weights s_e = exp(-(c_e - cmin) inv_gamma), inv_gamma = 1 / gamma.
// One pass of sums about the first elite c = p_0 (a point of the elite cloud,
// so the centred sums lose no digits to cancellation):
//   S = sum s_e,  d = sum s_e (p_e - c) / S,  T = sum s_e (p_e - c)(p_e - c)^T / S,
// then with pbar = c + d (the weighted elite mean), the new mean
// mu' = (1 - eta) mu + eta pbar and g = pbar - mu' = (1 - eta)(pbar - mu),
//   sum s_e (p_e - mu')(p_e - mu')^T / S = T - d d^T + g g^T,
// which is Eq. cov_update's weighted covariance about mu' exactly (in exact
// arithmetic).  Every sum runs on one warp: lane i adds the terms e = i,
// i + 32, ... in increasing order, then the lanes combine in a fixed butterfly,
// so the result does not depend on the block size.  float64 runs at 1/64 of
// the float32 rate here, and every dependent float64 operation is long: the
// mean and second-moment sums run in parallel, on different warps.  accum
// holds 2 + kMaxDp + kMaxDp^2 doubles.  With sig_copy (shared memory, leading
// dimension kMaxDp) the new covariance is also left there.
template <class PE, class CE>
__device__ void update_moments(PE p_e, CE c_e, double cmin, int q, int d_p, double inv_gamma,
                               double eta, double* mu, double* sigma, int ld, double* sw,
                               double* accum, double* sig_copy = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // the previous moments this thread combines, read while the weights are computed
  const bool combines = tid < d_p * d_p;
  const int ca_ = combines ? tid / d_p : 0, cb_ = combines ? tid % d_p : 0;
  const double mu_a = combines ? mu[ca_] : 0.0, mu_b = combines ? mu[cb_] : 0.0;
  const double sig_ab = combines ? sigma[ca_ * ld + cb_] : 0.0;
  const double mu_t = tid < d_p ? mu[tid] : 0.0;
  for (int e = tid; e < q; e += blockDim.x) sw[e] = exp(-(c_e(e) - cmin) * inv_gamma);
  __syncthreads();
  const int nsum = 1 + d_p + d_p * d_p;   // S, then d_p first and d_p^2 second moments
  for (int j = warp; j < nsum; j += nw) {
    double part = 0.0;
    if (j == 0) {
      for (int e = lane; e < q; e += 32) part += sw[e];
    } else if (j <= d_p) {
      const int a = j - 1;
      const double ca = p_e(0, a);
      for (int e = lane; e < q; e += 32) part += sw[e] * (p_e(e, a) - ca);
    } else {
      const int a = (j - 1 - d_p) / d_p, b = (j - 1 - d_p) % d_p;
      const double ca = p_e(0, a), cb = p_e(0, b);
      for (int e = lane; e < q; e += 32) part += sw[e] * (p_e(e, a) - ca) * (p_e(e, b) - cb);
    }
    part = warp_sum_f64(part);
    if (lane == 0) {
      accum[j] = part;
      if (j == 0) accum[nsum] = 1.0 / part;   // one float64 division for the update
    }
  }
  __syncthreads();
  const double inv_s = accum[nsum];
  // every read of the previous mu and sigma happened before the first barrier
  if (combines) {
    const int a = ca_, b = cb_;
    const double da = accum[1 + a] * inv_s, db = accum[1 + b] * inv_s;
    const double pa = p_e(0, a) + da, pb = p_e(0, b) + db;             // weighted means
    const double ga = (1.0 - eta) * (pa - mu_a), gb = (1.0 - eta) * (pb - mu_b);
    const double cov = accum[1 + d_p + tid] * inv_s - da * db + ga * gb;
    const double sig_new = (1.0 - eta) * sig_ab + eta * cov;
    sigma[a * ld + b] = sig_new;
    if (sig_copy != nullptr) sig_copy[a * kMaxDp + b] = sig_new;
    if (tid < d_p) mu[tid] = (1.0 - eta) * mu_t + eta * (p_e(0, tid) + accum[1 + tid] * inv_s);
  }
  __syncthreads();
}

// Lower Cholesky factor of sigma + eps I (d_p <= kMaxDp), single thread.  One
// reciprocal square root per column r = 1/sqrt(s): L_jj = s r, L_ij = v r
// (float64 division and square root are long instruction sequences here).
__device__ __forceinline__ void cholesky(const double* sigma, double eps, int d, double* L) {
  for (int i = 0; i < kMaxDp * kMaxDp; ++i) L[i] = 0.0;
  for (int jc = 0; jc < d; ++jc) {
    double s = sigma[jc * kMaxDp + jc] + eps;
    for (int k = 0; k < jc; ++k) s -= L[jc * kMaxDp + k] * L[jc * kMaxDp + k];
    const double rj = rsqrt(s);
    L[jc * kMaxDp + jc] = s * rj;
    for (int i = jc + 1; i < d; ++i) {
      double v = sigma[i * kMaxDp + jc];
      for (int k = 0; k < jc; ++k) v -= L[i * kMaxDp + k] * L[jc * kMaxDp + k];
      L[i * kMaxDp + jc] = v * rj;
    }
  }
}

// Cholesky factor of an imported state (plan_set_state) by the routine the
// selection kernels use, so that a resumed episode samples from the factor the
// interrupted one would have used, bit for bit.  One thread.
__global__ void import_chol_kernel(DevCem* cem, Params prm) {
  if (threadIdx.x == 0 && !cem->fresh) cholesky(cem->sigma, prm.cov_eps, prm.d_p, cem->chol);
}

__global__ void __launch_bounds__(kSelThreads)
select_update_kernel(const Layout* layout, DevCem* cem, int l, Params prm, const double* p,
                     const double* xi, const double* r, const double* cu, int* elite_out) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SelShared& sh = *reinterpret_cast<SelShared*>(shraw);
  pdl_wait();      // r, c_u, p and xi come from the solve kernel
  pdl_trigger();
  const int s = blockIdx.x;
  const Layout lay = layout[s];
  DevCem& st = cem[s];
  const int B = lay.B;
  if (B <= 0) return;
  const double* rs = r + lay.off;
  const double* cs = cu + lay.off;
  const int n_c = min(prm.n_c > 0 ? prm.n_c : 3 * prm.q, B);
  const int q = min(prm.q, n_c);
  select_constraint_set(rs, B, n_c, sh);
  select_elite_set(rs, cs, B, n_c, sh);
  const int d_p = prm.d_p;
  const double* ps = p + size_t(lay.off) * d_p;
  // indices are in [0, B) by construction; the clamp keeps every read in bounds
  auto id_of = [&](int e) { const int id = sh.idx[e]; return (id >= 0 && id < B) ? id : 0; };
  auto p_e = [&](int e, int a) { return ps[size_t(id_of(e)) * d_p + a]; };
  auto c_e = [&](int e) { return cs[id_of(e)] + rs[id_of(e)]; };
  update_moments(p_e, c_e, c_e(0), q, d_p, 1.0 / prm.gamma, prm.eta, st.mu, st.sigma, kMaxDp,
                 sh.sw, sh.acc);
  const int best = id_of(0);
  if (threadIdx.x == 0) {
    cholesky(st.sigma, prm.cov_eps, d_p, st.chol);
    st.best_index = best;
    st.best_r = rs[best];
    st.best_cu = cs[best];
    st.best_cost = cs[best] + rs[best];
    if (l == prm.L) { st.fresh = 0; st.step += 1ull; }
  }
  for (int a = threadIdx.x; a < d_p; a += blockDim.x) st.best_p[a] = ps[size_t(best) * d_p + a];
  for (int a = threadIdx.x; a < 2 * prm.n; a += blockDim.x)
    st.best_xi[a] = xi[size_t(lay.off + best) * 2 * prm.n + a];
  if (elite_out != nullptr)
    for (int e = threadIdx.x; e < q; e += blockDim.x) elite_out[size_t(s) * prm.q + e] = sh.idx[e];
}

__global__ void __launch_bounds__(kSelThreads)
select_only_kernel(const double* r, const double* cu, int B, int n_c, int q, int* elite) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SelShared& sh = *reinterpret_cast<SelShared*>(shraw);
  select_constraint_set(r, B, n_c, sh);
  select_elite_set(r, cu, B, n_c, sh);
  for (int e = threadIdx.x; e < q; e += blockDim.x) elite[e] = sh.idx[e];
}

__global__ void __launch_bounds__(kSelThreads)
update_only_kernel(const double* p_elite, const double* cost, int q, int d_p, double gamma,
                   double eta, double* mu, double* sigma) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SelShared& sh = *reinterpret_cast<SelShared*>(shraw);
  __shared__ double cmin;
  if (threadIdx.x == 0) {
    double c = cost[0];
    for (int e = 1; e < q; ++e) c = fmin(c, cost[e]);
    cmin = c;
  }
  __syncthreads();
  auto p_e = [&](int e, int a) { return p_elite[size_t(e) * d_p + a]; };
  auto c_e = [&](int e) { return cost[e]; };
  update_moments(p_e, c_e, cmin, q, d_p, 1.0 / gamma, eta, mu, sigma, d_p, sh.sw, sh.acc);
}

// ---------------------------------------------------------------------------
// Selection for B <= kSmallMaxB, one 256-thread block per scene: a bitonic
// sort of the (order key of r, sample index) pairs in shared memory gives the
// ConstraintEliteSet (its first n_c entries: n_c lowest r, ties to the lower
// index), and a second sort of the candidates by (order key of cu + r, sample
// index) gives the EliteSet in order.  The same sets as the large-B path.
constexpr int kSmallMaxB = 2048;
constexpr int kSmallMaxC = 1024;
constexpr int kSmallThreads = 256;
constexpr int kSmallPre = 128;           // elites whose p is staged in shared memory

struct SmallSel {
  unsigned long long key[kSmallMaxB];    // order keys of r, sorted in place
  int kidx[kSmallMaxB];                  // their sample indices
  unsigned long long ckey[kSmallMaxC];   // order keys of cu + r of the candidates
  unsigned ck32[kSmallMaxC];             // their upper 32 bits
  int idx[kSmallMaxC];                   // EliteSet, sorted by (cost, index)
  double sw[kSmallMaxC];
  double acc[kMaxDp * kMaxDp + kMaxDp + 2];
  double ce[kSmallMaxC];                 // costs c_u + r of the elites
  double pe[kSmallPre * kMaxDp];         // p of the first kSmallPre elites
  double bestv[2 + kMaxDp + 2 * kMaxCoef];   // best sample: r, c_u, p, xi
  double sig[kMaxDp * kMaxDp];           // the new covariance
  double inv_gamma;                      // 1 / gamma, taken while the elites are ranked
  double chol[kMaxDp * kMaxDp];          // its Cholesky factor
  int wsum[32];
  int total;
};

// Exclusive prefix sum over the block (blockDim.x <= 1024) of one count per
// thread, in thread order; *total is the block's sum.
__device__ void small_block_scan(int v, int* before, int* total, SmallSel& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh.wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nw ? sh.wsum[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) sh.wsum[lane] = wi - w;
    if (lane == 31) sh.total = wi;
  }
  __syncthreads();
  *before = sh.wsum[warp] + incl - v;
  *total = sh.total;
  __syncthreads();
}

__device__ __forceinline__ bool pair_gt(unsigned long long ka, int ia, unsigned long long kb,
                                        int ib) {
  return ka > kb || (ka == kb && ia > ib);
}

// One compare-exchange of the bitonic network at element e against its
// partner (ko, xo): e is the lower position when `lower`, and the kk-block of
// e sorts ascending when (e & kk) == 0.
__device__ __forceinline__ void bitonic_keep(unsigned long long& k, int& x, unsigned long long ko,
                                             int xo, bool lower, bool asc) {
  const bool gt = pair_gt(k, x, ko, xo);
  if (lower == asc ? gt : !gt) {
    k = ko;
    x = xo;
  }
}

// Stage at distance J < E between the elements of one thread.
template <int E, int J>
__device__ __forceinline__ void bitonic_intra(unsigned long long (&k)[E], int (&x)[E], int kk) {
#pragma unroll
  for (int u = 0; u < E; ++u) {
    if ((u & J) == 0) {
      const bool asc = ((E * int(threadIdx.x) + u) & kk) == 0;
      unsigned long long ka = k[u], kb = k[u ^ J];
      int xa = x[u], xb = x[u ^ J];
      if (pair_gt(ka, xa, kb, xb) == asc) {
        k[u] = kb; x[u] = xb;
        k[u ^ J] = ka; x[u ^ J] = xa;
      }
    }
  }
}

// Bitonic sort ascending by (key, idx) of P = 256 E pairs held E per thread,
// element E tid + u in k[u], x[u] (blockDim.x = 256).  Partners in the same
// thread are exchanged in registers, partners in the same warp by shuffles;
// only the stages whose partners sit in another warp (distance >= 32 E, six
// stages) go through the scratch arrays skey / sidx [P], laid out u-major so
// that those accesses are conflict-free.
template <int E>
__device__ void block_bitonic(unsigned long long (&k)[E], int (&x)[E], unsigned long long* skey,
                              int* sidx) {
  constexpr int P = 256 * E;
  const int tid = threadIdx.x;
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j < E) {
        if (j == 1) bitonic_intra<E, 1>(k, x, kk);
        if constexpr (E > 2) if (j == 2) bitonic_intra<E, (E > 2 ? 2 : 1)>(k, x, kk);
        if constexpr (E > 4) if (j == 4) bitonic_intra<E, (E > 4 ? 4 : 1)>(k, x, kk);
      } else if (j < 32 * E) {
        const int d = j / E;        // partner thread within the warp
        const bool lower = (tid & d) == 0;
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const unsigned long long ko = __shfl_xor_sync(0xffffffffu, k[u], d);
          const int xo = __shfl_xor_sync(0xffffffffu, x[u], d);
          bitonic_keep(k[u], x[u], ko, xo, lower, ((E * tid + u) & kk) == 0);
        }
      } else {
        const int d = j / E;        // partner thread in another warp
        __syncthreads();            // the previous exchange has been read
#pragma unroll
        for (int u = 0; u < E; ++u) {
          skey[u * 256 + tid] = k[u];
          sidx[u * 256 + tid] = x[u];
        }
        __syncthreads();
        const bool lower = (tid & d) == 0;
#pragma unroll
        for (int u = 0; u < E; ++u)
          bitonic_keep(k[u], x[u], skey[u * 256 + (tid ^ d)], sidx[u * 256 + (tid ^ d)], lower,
                       ((E * tid + u) & kk) == 0);
      }
    }
  }
  __syncthreads();   // the scratch arrays are free again
}

// ConstraintEliteSet (the n_c lowest (r key, index)) staged in sh.ckey /
// sh.idx [0..n_c), padded to P2 (a power of two, >= 256).
template <int E>
__device__ void small_constraint_set(const double* r, const double* cu, int B, int n_c, int P2,
                                     SmallSel& sh) {
  unsigned long long k[E];
  int x[E];
  double c[E];      // c_u, loaded with r so that both latencies overlap
  const int tid = threadIdx.x;
#pragma unroll
  for (int u = 0; u < E; ++u) {
    const int e = E * tid + u;
    k[u] = e < B ? ord_key(r[e]) : ~0ull;    // padding sorts last
    c[u] = e < B ? cu[e] : 0.0;
    x[u] = e;
  }
  // Feasible samples score exactly r = 0, the smallest possible r (a sum of
  // max(0, .) terms).  When at least n_c of them exist, the n_c lowest
  // (key, index) pairs are the n_c zero-score samples of lowest index: a
  // block-wide compaction in index order gives the same set as the sort.
  // Their cost key is that of c_u alone: with r = +-0, c_u + r has the key
  // of c_u (keys take -0 as +0 and every NaN as one).
  const unsigned long long kzero = ord_key(0.0);
  int nzero = 0;
#pragma unroll
  for (int u = 0; u < E; ++u) nzero += k[u] == kzero ? 1 : 0;
  int before = 0, total = 0;
  small_block_scan(nzero, &before, &total, sh);
  const bool zero_set = total >= n_c;      // block-uniform
  if (!zero_set) block_bitonic<E>(k, x, sh.key, sh.kidx);
#pragma unroll
  for (int u = 0; u < E; ++u) {
    // position in the set: the rank among zero scores, or the sorted position
    int e = E * tid + u;
    if (zero_set) e = k[u] == kzero ? before++ : n_c;
    if (e < n_c) {
      const unsigned long long kc = zero_set ? ord_key(c[u]) : ord_key(cu[x[u]] + r[x[u]]);
      sh.ckey[e] = kc;
      sh.ck32[e] = unsigned(kc >> 32);
      sh.idx[e] = x[u];
    }
  }
  for (int e = n_c + tid; e < P2; e += blockDim.x) {
    sh.ckey[e] = ~0ull;
    sh.ck32[e] = ~0u;
    sh.idx[e] = B + e;
  }
  __syncthreads();
}

// EliteSet: the candidates sorted by (cost key, index), the first q into sh.idx.
template <int E>
__device__ void small_elite_set(int q, SmallSel& sh) {
  unsigned long long k[E];
  int x[E];
  const int tid = threadIdx.x;
#pragma unroll
  for (int u = 0; u < E; ++u) {
    k[u] = sh.ckey[E * tid + u];
    x[u] = sh.idx[E * tid + u];
  }
  block_bitonic<E>(k, x, sh.key, sh.kidx);   // ends with a barrier: sh.idx is free
#pragma unroll
  for (int u = 0; u < E; ++u)
    if (E * tid + u < q) sh.idx[E * tid + u] = x[u];
  __syncthreads();
}

// ConstraintEliteSet, then the EliteSet sorted into sh.idx[0..q) (blockDim.x = 256).
__device__ void small_elites(const double* r, const double* cu, int B, int n_c, int q,
                             SmallSel& sh) {
  int P = 256;
  while (P < B) P <<= 1;
  int P2 = 256;
  while (P2 < n_c) P2 <<= 1;
  switch (P) {
    case 256: small_constraint_set<1>(r, cu, B, n_c, P2, sh); break;
    case 512: small_constraint_set<2>(r, cu, B, n_c, P2, sh); break;
    case 1024: small_constraint_set<4>(r, cu, B, n_c, P2, sh); break;
    default: small_constraint_set<8>(r, cu, B, n_c, P2, sh); break;
  }
  if (n_c <= 256) {
    // few candidates: each one's rank is the number of (cost key, index)
    // pairs below it (no barriers); ranks are distinct since indices are.
    // The upper 32 bits of the keys order all pairs whose upper halves
    // differ (four per 16-byte load); only candidates that share their upper
    // half with another compare the full pairs.  Entries n_c..P2-1 hold the
    // largest upper half and never count.
    const int tid = threadIdx.x;
    if (tid < n_c) {
      const unsigned long long kc = sh.ckey[tid];
      const unsigned k32 = unsigned(kc >> 32);
      const int ic = sh.idx[tid];
      const uint4* c4 = reinterpret_cast<const uint4*>(sh.ck32);
      int lt0 = 0, lt1 = 0, eq = 0;
      for (int h4 = 0; h4 < (n_c + 3) / 4; ++h4) {
        const uint4 a = c4[h4];
        lt0 += (a.x < k32 ? 1 : 0) + (a.y < k32 ? 1 : 0);
        lt1 += (a.z < k32 ? 1 : 0) + (a.w < k32 ? 1 : 0);
        eq += (a.x == k32 ? 1 : 0) + (a.y == k32 ? 1 : 0) + (a.z == k32 ? 1 : 0) +
              (a.w == k32 ? 1 : 0);
      }
      int rank = lt0 + lt1;
      if (eq > 1)      // another candidate shares the upper half (itself counts once)
        for (int h = 0; h < n_c; ++h)
          if (sh.ck32[h] == k32) rank += pair_gt(kc, ic, sh.ckey[h], sh.idx[h]) ? 1 : 0;
      if (rank < q) sh.kidx[rank] = ic;
    }
    __syncthreads();
    for (int e = tid; e < q; e += blockDim.x) sh.idx[e] = sh.kidx[e];
    __syncthreads();
    return;
  }
  switch (P2) {
    case 512: small_elite_set<2>(q, sh); break;
    default: small_elite_set<4>(q, sh); break;
  }
}

// one block per SM is all it needs: the explicit bound lets ptxas use the
// registers it wants (its default for 256 threads spilled)
__global__ void __launch_bounds__(kSmallThreads, 1)
select_update_small_kernel(const Layout* layout, DevCem* cem, int l, Params prm, const double* p,
                           const double* xi, const double* r, const double* cu, int* elite_out) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SmallSel& sh = *reinterpret_cast<SmallSel*>(shraw);
  pdl_wait();      // r, c_u, p and xi come from the solve kernel
  pdl_trigger();
  const int s = blockIdx.x;
  const Layout lay = layout[s];
  DevCem& st = cem[s];
  const int B = lay.B;
  if (B <= 0) return;
  const double* rs = r + lay.off;
  const double* cs = cu + lay.off;
  const int n_c = min(prm.n_c > 0 ? prm.n_c : 3 * prm.q, B);
  const int q = min(prm.q, n_c);
  small_elites(rs, cs, B, n_c, q, sh);
  const int d_p = prm.d_p;
  const double* ps = p + size_t(lay.off) * d_p;
  auto id_of = [&](int e) { const int id = sh.idx[e]; return (id >= 0 && id < B) ? id : 0; };
  // one parallel gather of everything the update and the best pair read (the
  // elites' costs, the first kSmallPre elites' p, the best sample's r, c_u, p
  // and xi), so that their global-memory latencies overlap
  const int best = id_of(0);
  const int qp = min(q, kSmallPre);
  const int nx = 2 * prm.n;
  const int n_gather = q + qp * d_p + 2 + d_p + nx;
  for (int t = threadIdx.x; t < n_gather; t += blockDim.x) {
    if (t < q) {
      sh.ce[t] = cs[id_of(t)] + rs[id_of(t)];
    } else if (t < q + qp * d_p) {
      const int tt = t - q;
      sh.pe[tt] = ps[size_t(id_of(tt / d_p)) * d_p + tt % d_p];
    } else {
      const int b = t - q - qp * d_p;
      sh.bestv[b] = b == 0 ? rs[best]
                  : b == 1 ? cs[best]
                  : b < 2 + d_p ? ps[size_t(best) * d_p + (b - 2)]
                                : xi[size_t(lay.off + best) * nx + (b - 2 - d_p)];
    }
  }
  // the last thread (idle in the gather when it is short) takes 1 / gamma
  if (threadIdx.x == blockDim.x - 1) sh.inv_gamma = 1.0 / prm.gamma;
  __syncthreads();
  auto p_e = [&](int e, int a) {
    return e < kSmallPre ? sh.pe[e * d_p + a] : ps[size_t(id_of(e)) * d_p + a];
  };
  auto c_e = [&](int e) { return sh.ce[e]; };
  update_moments(p_e, c_e, c_e(0), q, d_p, sh.inv_gamma, prm.eta, st.mu, st.sigma, kMaxDp, sh.sw,
                 sh.acc, sh.sig);
  // the factorisation reads the covariance from shared memory and its factor
  // is written out by the whole block
  if (threadIdx.x == 0) cholesky(sh.sig, prm.cov_eps, d_p, sh.chol);
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxDp * kMaxDp; i += blockDim.x) st.chol[i] = sh.chol[i];
  if (threadIdx.x == 0) {
    st.best_index = best;
    st.best_r = sh.bestv[0];
    st.best_cu = sh.bestv[1];
    st.best_cost = sh.bestv[1] + sh.bestv[0];
    if (l == prm.L) { st.fresh = 0; st.step += 1ull; }
  }
  for (int a = threadIdx.x; a < d_p; a += blockDim.x) st.best_p[a] = sh.bestv[2 + a];
  for (int a = threadIdx.x; a < nx; a += blockDim.x) st.best_xi[a] = sh.bestv[2 + d_p + a];
  if (elite_out != nullptr)
    for (int e = threadIdx.x; e < q; e += blockDim.x) elite_out[size_t(s) * prm.q + e] = sh.idx[e];
}

__global__ void __launch_bounds__(kSmallThreads)
select_only_small_kernel(const double* r, const double* cu, int B, int n_c, int q, int* elite) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SmallSel& sh = *reinterpret_cast<SmallSel*>(shraw);
  small_elites(r, cu, B, n_c, q, sh);
  for (int e = threadIdx.x; e < q; e += blockDim.x) elite[e] = sh.idx[e];
}

// Per-slot states from / to a table of episode states: dst[s] = src[idx[s]]
// for idx[s] >= 0 (gather) or dst[idx[s]] = src[s] (scatter).
__global__ void cem_copy_kernel(DevCem* dst, const DevCem* src, const int* idx, int S, int scatter) {
  constexpr int W = sizeof(DevCem) / sizeof(unsigned long long);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= S * W) return;
  const int s = e / W, w = e % W;
  const int r = idx[s];
  if (r < 0) return;
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(scatter ? src + s : src + r);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(scatter ? dst + r : dst + s);
  b[w] = a[w];
}

// One MPC cycle through host buffers: the host writes the scene record, its
// obstacle rows and the sampling state into a pinned host buffer mapped into
// the device's address space; these kernels move them in 8-byte words at the
// head of the cycle's graph and move the final state (with the best pair) and
// the timeout flag back at its tail.  Offsets are in words; the host sizes the
// obstacle region for max_obs rows and checks n_obs <= max_obs before staging.
__global__ void io_in_kernel(const unsigned long long* io, size_t w_obs, size_t w_cem,
                             DevScene* scene, double* obs, DevCem* cem, Params prm) {
  constexpr int WS = sizeof(DevScene) / sizeof(unsigned long long);
  constexpr int WC = sizeof(DevCem) / sizeof(unsigned long long);
  const int n_obs_w = reinterpret_cast<const DevScene*>(io)->n_obs * 6;
  unsigned long long* ds = reinterpret_cast<unsigned long long*>(scene);
  unsigned long long* dob = reinterpret_cast<unsigned long long*>(obs);
  unsigned long long* dc = reinterpret_cast<unsigned long long*>(cem);
  for (int i = threadIdx.x; i < WS; i += blockDim.x) ds[i] = io[i];
  for (int i = threadIdx.x; i < n_obs_w; i += blockDim.x) dob[i] = io[w_obs + i];
  for (int i = threadIdx.x; i < WC; i += blockDim.x) dc[i] = io[w_cem + i];
  // a warm start's covariance is factored here by the selection kernels'
  // routine, so that the cycle samples exactly as one that kept its state on
  // the device would
  __syncthreads();
  if (threadIdx.x == 0 && !cem->fresh) cholesky(cem->sigma, prm.cov_eps, prm.d_p, cem->chol);
}

__global__ void io_out_kernel(const DevCem* cem, const int* tc_err, unsigned long long* io,
                              size_t w_ret) {
  constexpr int WC = sizeof(DevCem) / sizeof(unsigned long long);
  const unsigned long long* sc = reinterpret_cast<const unsigned long long*>(cem);
  for (int i = threadIdx.x; i < WC; i += blockDim.x) io[w_ret + i] = sc[i];
  if (threadIdx.x == 0) io[w_ret + WC] = static_cast<unsigned long long>(*tc_err != 0);
  __threadfence_system();
}

}  // namespace

cudaError_t launch_cem_copy(DevCem* dst, const DevCem* src, const int* idx, int S, bool scatter,
                            cudaStream_t s) {
  if (S == 0) return cudaSuccess;
  constexpr int W = sizeof(DevCem) / sizeof(unsigned long long);
  cem_copy_kernel<<<(S * W + 255) / 256, 256, 0, s>>>(dst, src, idx, S, scatter ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevScene* scenes, const Layout* layout, const DevCem* cem, int S,
                          int max_B, int l, const Params& prm, double* p, cudaStream_t s,
                          bool pdl, const double* zbuf) {
  if (S == 0 || max_B == 0) return cudaSuccess;
  dim3 grid((max_B + 127) / 128, S);
  if (!pdl) {
    sample_kernel<<<grid, 128, 0, s>>>(scenes, layout, cem, l, prm, zbuf, p);
    return cudaGetLastError();
  }
  return launch_pdl(sample_kernel, grid, dim3(128), 0, s, scenes, layout, cem, l, prm, zbuf, p);
}

cudaError_t launch_import_chol(DevCem* cem, const Params& prm, cudaStream_t s) {
  import_chol_kernel<<<1, 32, 0, s>>>(cem, prm);
  return cudaGetLastError();
}

cudaError_t launch_normals(const Layout* layout, const DevCem* cem, int S, int max_B, int l,
                           const Params& prm, double* zbuf, cudaStream_t s) {
  if (S == 0 || max_B == 0) return cudaSuccess;
  dim3 grid((max_B + 127) / 128, S);
  normals_kernel<<<grid, 128, 0, s>>>(layout, cem, l, prm, zbuf);
  return cudaGetLastError();
}

cudaError_t launch_io_in(const void* io, size_t o_obs, size_t o_cem, DevScene* scene, double* obs,
                         DevCem* cem, const Params& prm, cudaStream_t s) {
  io_in_kernel<<<1, 256, 0, s>>>(static_cast<const unsigned long long*>(io), o_obs / 8, o_cem / 8,
                                 scene, obs, cem, prm);
  return cudaGetLastError();
}

cudaError_t launch_io_out(const DevCem* cem, const int* tc_err, void* io, size_t o_ret,
                          cudaStream_t s) {
  io_out_kernel<<<1, 256, 0, s>>>(cem, tc_err, static_cast<unsigned long long*>(io), o_ret / 8);
  return cudaGetLastError();
}

// Shared-memory attributes of the selection kernels, set once per device
// (a function attribute applies to the current device only).
static std::atomic<bool> g_sel_attr[64];
static void sel_attr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    dev = 0;
  }
  if (g_sel_attr[dev].load()) return;
  cudaFuncSetAttribute(select_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(select_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(update_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(select_update_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SmallSel)));
  cudaFuncSetAttribute(select_only_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SmallSel)));
  g_sel_attr[dev].store(true);
}

cudaError_t launch_select_update(const Layout* layout, DevCem* cem, int S, int l,
                                 const Params& prm, const double* p, const double* xi,
                                 const double* r, const double* cu, int* elite_out,
                                 int max_B, cudaStream_t s) {
  if (S == 0) return cudaSuccess;
  sel_attr();
  if (max_B <= kSmallMaxB && (prm.n_c > 0 ? prm.n_c : 3 * prm.q) <= kSmallMaxC) {
    return launch_pdl(select_update_small_kernel, dim3(S), dim3(kSmallThreads), sizeof(SmallSel),
                      s, layout, cem, l, prm, p, xi, r, cu, elite_out);
  }
  return launch_pdl(select_update_kernel, dim3(S), dim3(kSelThreads), sizeof(SelShared), s, layout,
                    cem, l, prm, p, xi, r, cu, elite_out);
}

cudaError_t launch_select_only(const double* r, const double* cu, int B, int n_c, int q,
                               int* elite, cudaStream_t s) {
  sel_attr();
  if (B <= kSmallMaxB && n_c <= kSmallMaxC) {
    select_only_small_kernel<<<1, kSmallThreads, sizeof(SmallSel), s>>>(r, cu, B, n_c, q, elite);
    return cudaGetLastError();
  }
  select_only_kernel<<<1, kSelThreads, sizeof(SelShared), s>>>(r, cu, B, n_c, q, elite);
  return cudaGetLastError();
}

cudaError_t launch_update_only(const double* p_elite, const double* cost, int q, int d_p,
                               double gamma, double eta, double* mu, double* sigma,
                               cudaStream_t s) {
  sel_attr();
  update_only_kernel<<<1, kSelThreads, sizeof(SelShared), s>>>(p_elite, cost, q, d_p, gamma, eta,
                                                               mu, sigma);
  return cudaGetLastError();
}

void cem_setup() { sel_attr(); }

}  // namespace plan

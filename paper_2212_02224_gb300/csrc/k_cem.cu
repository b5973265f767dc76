// Outer loop of Alg. 1 on the device: sampling (line 4), ConstraintEliteSet and
// EliteSet (lines 10-13), and the distribution update of Eqs. (mean_update,
// cov_update, s_formula), one thread block per scene, float64.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
// key = (seed_lo, seed_hi) and counter = (j, l | c << 16, step_lo, step_hi);
// Box-Muller turns word pairs (2q, 2q+1) into normals.
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

// Alg. 1 line 4 for every scene: grid (ceil(max_B / 128), S).
__global__ void sample_kernel(const DevScene* scenes, const Layout* layout, const DevCem* cem,
                              int l, Params prm, double* p) {
  const int s = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const Layout lay = layout[s];
  if (j >= lay.B) return;
  const DevCem& st = cem[s];
  const int d_p = prm.d_p, ns = prm.n_seg;
  unsigned w[kMaxDp];
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
  double* out = p + size_t(lay.off + j) * d_p;
  if (l == 1 && st.fresh) {
    const DevScene& sc = scenes[s];
    for (int e = 0; e < ns; ++e) {
      int idx = int(floor(unit_open(w[e]) * sc.n_lanes));
      if (idx > sc.n_lanes - 1) idx = sc.n_lanes - 1;
      out[e] = (idx + 0.5) * sc.lane_width;
    }
    for (int e = ns; e < 2 * ns; ++e)
      out[e] = prm.v_des_lo + (prm.v_des_hi - prm.v_des_lo) * unit_open(w[e]);
  } else {
    double z[kMaxDp];
    for (int q = 0; 2 * q < d_p; ++q) {
      const double r = sqrt(-2.0 * log(unit_open(w[2 * q])));
      const double th = 2.0 * CUDART_PI * unit_open(w[2 * q + 1]);
      z[2 * q] = r * cos(th);
      z[2 * q + 1] = r * sin(th);
    }
    for (int a = 0; a < d_p; ++a) {
      double v = 0.0;
      for (int b = 0; b <= a; ++b) v += z[b] * st.chol[a * kMaxDp + b];
      out[a] = st.mu[a] + v;
    }
  }
}

// Total order on doubles: -0 is +0, NaN sorts after everything.
__device__ __forceinline__ unsigned long long ord_key(double v) {
  if (v != v) return 0xfff8000000000000ull;   // canonical NaN, after +inf
  if (v == 0.0) v = 0.0;
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
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
  double acc[kMaxDp * kMaxDp + kMaxDp + 1];
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

// Eqs. (mean_update, cov_update, s_formula) over the q elites p_e(e), costs c_e(e).
template <class PE, class CE>
__device__ void update_moments(PE p_e, CE c_e, double cmin, int q, int d_p, double gamma,
                               double eta, double* mu, double* sigma, int ld, SelShared& sh) {
  const int tid = threadIdx.x;
  for (int e = tid; e < q; e += blockDim.x) sh.sw[e] = exp(-(c_e(e) - cmin) / gamma);
  __syncthreads();
  double* mu_new = sh.acc;
  double* ssum = sh.acc + kMaxDp;
  if (tid == 0) {
    double S = 0.0;
    for (int e = 0; e < q; ++e) S += sh.sw[e];
    *ssum = S;
  }
  __syncthreads();
  if (tid < d_p) {
    double a = 0.0;
    for (int e = 0; e < q; ++e) a += sh.sw[e] * p_e(e, tid);
    mu_new[tid] = (1.0 - eta) * mu[tid] + eta * a / *ssum;
  }
  __syncthreads();
  if (tid < d_p * d_p) {
    const int a = tid / d_p, b = tid % d_p;
    double acc = 0.0;
    for (int e = 0; e < q; ++e)
      acc += sh.sw[e] * (p_e(e, a) - mu_new[a]) * (p_e(e, b) - mu_new[b]);
    sigma[a * ld + b] = (1.0 - eta) * sigma[a * ld + b] + eta * acc / *ssum;
  }
  __syncthreads();
  if (tid < d_p) mu[tid] = mu_new[tid];
  __syncthreads();
}

// Lower Cholesky factor of sigma + eps I (d_p <= 8), single thread.
__device__ void cholesky(const double* sigma, double eps, int d, double* L) {
  for (int i = 0; i < kMaxDp * kMaxDp; ++i) L[i] = 0.0;
  for (int jc = 0; jc < d; ++jc) {
    double s = sigma[jc * kMaxDp + jc] + eps;
    for (int k = 0; k < jc; ++k) s -= L[jc * kMaxDp + k] * L[jc * kMaxDp + k];
    const double dj = sqrt(s);
    L[jc * kMaxDp + jc] = dj;
    for (int i = jc + 1; i < d; ++i) {
      double v = sigma[i * kMaxDp + jc];
      for (int k = 0; k < jc; ++k) v -= L[i * kMaxDp + k] * L[jc * kMaxDp + k];
      L[i * kMaxDp + jc] = v / dj;
    }
  }
}

__global__ void __launch_bounds__(kSelThreads)
select_update_kernel(const Layout* layout, DevCem* cem, int l, Params prm, const double* p,
                     const double* xi, const double* r, const double* cu, int* elite_out) {
  extern __shared__ __align__(16) unsigned char shraw[];
  SelShared& sh = *reinterpret_cast<SelShared*>(shraw);
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
  update_moments(p_e, c_e, c_e(0), q, d_p, prm.gamma, prm.eta, st.mu, st.sigma, kMaxDp, sh);
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
  update_moments(p_e, c_e, cmin, q, d_p, gamma, eta, mu, sigma, d_p, sh);
}

// ---------------------------------------------------------------------------
// Warp-per-scene selection for B <= kWarpMaxB: the same ConstraintEliteSet /
// EliteSet and distribution update as the block kernels above, with only
// warp-level synchronisation.  Keys live in shared memory (per warp).
constexpr int kWarpMaxB = 2048;
constexpr int kWarpMaxC = 1024;
constexpr int kWarpsPerCta = 4;

struct WarpSel {
  unsigned long long key[kWarpMaxB];   // order keys of r, then of the candidates' costs
  int cand[kWarpMaxC];
  unsigned hist[256];
  double sw[kWarpMaxC];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ConstraintEliteSet of one scene into ws.cand[0..n_c) (increasing index order).
__device__ void warp_constraint_set(const double* r, int B, int n_c, WarpSel& ws) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < B; i += 32) ws.key[i] = ord_key(r[i]);
  __syncwarp();
  unsigned long long prefix = 0ull;
  int need = n_c;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int d = lane; d < 256; d += 32) ws.hist[d] = 0u;
    __syncwarp();
    for (int i = lane; i < B; i += 32) {
      const unsigned long long k = ws.key[i];
      if (shift == 56 || ((k ^ prefix) >> (shift + 8)) == 0ull)
        atomicAdd(&ws.hist[(k >> shift) & 255ull], 1u);
    }
    __syncwarp();
    unsigned loc = 0;
    for (int d = 0; d < 8; ++d) loc += ws.hist[8 * lane + d];
    unsigned incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, incl >= unsigned(need));
    const int first = __ffs(hit) - 1;
    int digit = 0, cum = 0;
    if (lane == first) {
      unsigned c = incl - loc;
      int d = 8 * lane;
      for (; d < 8 * lane + 7; ++d) {
        if (c + ws.hist[d] >= unsigned(need)) break;
        c += ws.hist[d];
      }
      digit = d;
      cum = int(c);
    }
    digit = __shfl_sync(0xffffffffu, digit, first < 0 ? 0 : first);
    cum = __shfl_sync(0xffffffffu, cum, first < 0 ? 0 : first);
    need -= cum;
    prefix |= static_cast<unsigned long long>(digit) << shift;
    __syncwarp();
  }
  const unsigned long long T = prefix;
  const unsigned lt = (1u << lane) - 1u;
  int ties = 0, sel = 0;
  for (int base = 0; base < B; base += 32) {
    const int i = base + lane;
    const unsigned long long k = i < B ? ws.key[i] : ~0ull;
    const bool less = i < B && k < T, eq = i < B && k == T;
    const unsigned em = __ballot_sync(0xffffffffu, eq);
    const bool take = less || (eq && ties + __popc(em & lt) < need);
    const unsigned tm = __ballot_sync(0xffffffffu, take);
    const int pos = sel + __popc(tm & lt);
    if (take && pos < n_c) ws.cand[pos] = i;
    ties += __popc(em);
    sel += __popc(tm);
  }
  __syncwarp();
}

// EliteSet: the candidates sorted by (cu + r, index) into ws.cand[0..n_c).
__device__ void warp_elite_sort(const double* r, const double* cu, int B, int n_c, WarpSel& ws) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < n_c) P <<= 1;
  for (int i = lane; i < P; i += 32) {
    const int id = i < n_c ? ws.cand[i] : -1;
    if (id >= 0 && id < B) {
      ws.key[i] = ord_key(cu[id] + r[id]);
    } else {
      ws.key[i] = ~0ull;
      ws.cand[i] = 0x7fffffff;
    }
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool asc = (i & k) == 0;
          const unsigned long long ka = ws.key[i], kb = ws.key[ixj];
          const int ia = ws.cand[i], ib = ws.cand[ixj];
          const bool gt = (ka > kb) || (ka == kb && ia > ib);
          if (gt == asc) {
            ws.key[i] = kb; ws.key[ixj] = ka;
            ws.cand[i] = ib; ws.cand[ixj] = ia;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(32 * kWarpsPerCta)
select_update_warp_kernel(const Layout* layout, DevCem* cem, int S, int l, Params prm,
                          const double* p, const double* xi, const double* r, const double* cu,
                          int* elite_out) {
  extern __shared__ __align__(16) unsigned char shraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kWarpsPerCta + warp;
  if (s >= S) return;
  WarpSel& ws = reinterpret_cast<WarpSel*>(shraw)[warp];
  const Layout lay = layout[s];
  DevCem& st = cem[s];
  const int B = lay.B;
  if (B <= 0) return;
  const double* rs = r + lay.off;
  const double* cs = cu + lay.off;
  const int n_c = min(prm.n_c > 0 ? prm.n_c : 3 * prm.q, B);
  const int q = min(prm.q, n_c);
  warp_constraint_set(rs, B, n_c, ws);
  warp_elite_sort(rs, cs, B, n_c, ws);
  const int d_p = prm.d_p;
  const double* ps = p + size_t(lay.off) * d_p;
  auto id_of = [&](int e) { const int id = ws.cand[e]; return (id >= 0 && id < B) ? id : 0; };
  // Eqs. (mean_update, cov_update, s_formula), lanes over elites
  const double cmin = cs[id_of(0)] + rs[id_of(0)];
  for (int e = lane; e < q; e += 32) {
    const int id = id_of(e);
    ws.sw[e] = exp(-(cs[id] + rs[id] - cmin) / prm.gamma);
  }
  __syncwarp();
  double part = 0.0;
  for (int e = lane; e < q; e += 32) part += ws.sw[e];
  const double Ssum = warp_sum(part);
  double mu_new[kMaxDp];
  for (int a = 0; a < d_p; ++a) {
    double v = 0.0;
    for (int e = lane; e < q; e += 32) v += ws.sw[e] * ps[size_t(id_of(e)) * d_p + a];
    mu_new[a] = (1.0 - prm.eta) * st.mu[a] + prm.eta * warp_sum(v) / Ssum;
  }
  double sg_new[kMaxDp * kMaxDp];
  for (int a = 0; a < d_p; ++a) {
    for (int b = 0; b < d_p; ++b) {
      double v = 0.0;
      for (int e = lane; e < q; e += 32) {
        const double* pe = ps + size_t(id_of(e)) * d_p;
        v += ws.sw[e] * (pe[a] - mu_new[a]) * (pe[b] - mu_new[b]);
      }
      sg_new[a * kMaxDp + b] = (1.0 - prm.eta) * st.sigma[a * kMaxDp + b] + prm.eta * warp_sum(v) / Ssum;
    }
  }
  __syncwarp();
  const int best = id_of(0);
  if (lane == 0) {
    for (int a = 0; a < d_p; ++a) {
      st.mu[a] = mu_new[a];
      for (int b = 0; b < d_p; ++b) st.sigma[a * kMaxDp + b] = sg_new[a * kMaxDp + b];
    }
    cholesky(st.sigma, prm.cov_eps, d_p, st.chol);
    st.best_index = best;
    st.best_r = rs[best];
    st.best_cu = cs[best];
    st.best_cost = cs[best] + rs[best];
    if (l == prm.L) { st.fresh = 0; st.step += 1ull; }
  }
  for (int a = lane; a < d_p; a += 32) st.best_p[a] = ps[size_t(best) * d_p + a];
  for (int a = lane; a < 2 * prm.n; a += 32) st.best_xi[a] = xi[size_t(lay.off + best) * 2 * prm.n + a];
  if (elite_out != nullptr)
    for (int e = lane; e < q; e += 32) elite_out[size_t(s) * prm.q + e] = ws.cand[e];
}

__global__ void __launch_bounds__(32)
select_only_warp_kernel(const double* r, const double* cu, int B, int n_c, int q, int* elite) {
  extern __shared__ __align__(16) unsigned char shraw[];
  WarpSel& ws = *reinterpret_cast<WarpSel*>(shraw);
  warp_constraint_set(r, B, n_c, ws);
  warp_elite_sort(r, cu, B, n_c, ws);
  for (int e = threadIdx.x; e < q; e += 32) elite[e] = ws.cand[e];
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

}  // namespace

cudaError_t launch_cem_copy(DevCem* dst, const DevCem* src, const int* idx, int S, bool scatter,
                            cudaStream_t s) {
  if (S == 0) return cudaSuccess;
  constexpr int W = sizeof(DevCem) / sizeof(unsigned long long);
  cem_copy_kernel<<<(S * W + 255) / 256, 256, 0, s>>>(dst, src, idx, S, scatter ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevScene* scenes, const Layout* layout, const DevCem* cem, int S,
                          int max_B, int l, const Params& prm, double* p, cudaStream_t s) {
  if (S == 0 || max_B == 0) return cudaSuccess;
  dim3 grid((max_B + 127) / 128, S);
  sample_kernel<<<grid, 128, 0, s>>>(scenes, layout, cem, l, prm, p);
  return cudaGetLastError();
}

static bool g_sel_attr = false;
static void sel_attr() {
  if (g_sel_attr) return;
  cudaFuncSetAttribute(select_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(select_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(update_only_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(SelShared)));
  cudaFuncSetAttribute(select_update_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(WarpSel) * kWarpsPerCta));
  cudaFuncSetAttribute(select_only_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(sizeof(WarpSel)));
  g_sel_attr = true;
}

cudaError_t launch_select_update(const Layout* layout, DevCem* cem, int S, int l,
                                 const Params& prm, const double* p, const double* xi,
                                 const double* r, const double* cu, int* elite_out,
                                 int max_B, cudaStream_t s) {
  if (S == 0) return cudaSuccess;
  sel_attr();
  if (max_B <= kWarpMaxB && (prm.n_c > 0 ? prm.n_c : 3 * prm.q) <= kWarpMaxC) {
    select_update_warp_kernel<<<(S + kWarpsPerCta - 1) / kWarpsPerCta, 32 * kWarpsPerCta,
                                sizeof(WarpSel) * kWarpsPerCta, s>>>(layout, cem, S, l, prm, p, xi,
                                                                     r, cu, elite_out);
    return cudaGetLastError();
  }
  select_update_kernel<<<S, kSelThreads, sizeof(SelShared), s>>>(layout, cem, l, prm, p, xi, r, cu,
                                                                 elite_out);
  return cudaGetLastError();
}

cudaError_t launch_select_only(const double* r, const double* cu, int B, int n_c, int q,
                               int* elite, cudaStream_t s) {
  sel_attr();
  if (B <= kWarpMaxB && n_c <= kWarpMaxC) {
    select_only_warp_kernel<<<1, 32, sizeof(WarpSel), s>>>(r, cu, B, n_c, q, elite);
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

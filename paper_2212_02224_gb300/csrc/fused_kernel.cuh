// Fused FP32 lower-level solve (kernel template, included by k_fused.cu and
// k_fused_road.cu): Step 1 (Alg. 1 line 7 through the folded KKT
// inverse of Eq. over_3), all K iterations of Alg. 2 and the scoring of
// Alg. 1 line 9 / Sec. V-A, 1, 2 or 4 warps per sample, all state on chip.
// Two launch forms run the same per-sample code (solve_sample): one tile of
// samples per CTA (fused_kernel), or one wave of CTAs whose sample groups
// take samples from a device counter (fused_persistent_kernel).  Products
// whose rounding the compiler could otherwise contract in two ways are written
// as explicit fmaf, so both forms give the same bits.
//
// State is kept relative to the Step-1 solution: delta = xi - xi_bar.  Per
// iteration and sample the warp(s)
//   A. evaluates x, y and their derivatives at the lane's timesteps (slot
//      mapping below) as (reference at xi_bar) + W delta (Eq. param; basis
//      rows staged in shared memory),
//   B. projects onto every obstacle ellipse (Eqs. split_alpha_o, clip_d_o),
//   C. projects velocity and acceleration (Eqs. clip_d_v, clip_d_a), the lane
//      rows (Eq. update_slack) and accumulates the transposed contraction
//        w = F^T (h - F xi) + G^T (e - s - G xi),
//   D. reduce-scatters w over the warp, updates the multipliers
//      lambda += rho/2 w (Eq. update_lagrange) and takes the xi-step of
//      Eq. split_xy in increment form
//        delta' = delta + M (lambda + rho w - delta).
// The increment form is exact: with H = I + rho P, P = F^T F + G^T G and the
// KKT inverse [[M, C], [C^T, D]] of [[H, A^T], [A, 0]], M H = I - C A, so
// M (xi_bar + lambda + rho F^T h + rho G^T (e - s)) + C b0
//   = xi + M (xi_bar - xi + lambda + rho w) + C (b0 - A xi),
// and every iterate satisfies A xi = b0.  Working on delta (metres) instead
// of xi (hundreds of metres) keeps float32 rounding from accumulating.
//
// The closed form of Eq. split_alpha_o is used without trigonometry: for an
// obstacle with scaled offset (sx, sy) = ((x - x_o)/a, (y - y_o)/b) and
// d^2 = sx^2 + sy^2, cos(alpha) = sx/d, sin(alpha) = sy/d, so the clipped
// point h = o + (a max(1,d) cos, b max(1,d) sin) differs from the trajectory
// point by (x - x_o, y - y_o) (1/d - 1) when d < 1 and by zero otherwise.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"

namespace plan {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// MUFU reciprocal square root and approximate division with subnormals flushed:
// without the .ftz forms the compiler wraps each MUFU operation in a subnormal
// range fix-up, which cost about 6 % of the solve at B = 1000.  Callers treat
// operands below FLT_MIN as zero (a squared speed, acceleration or scaled
// distance below 1.2e-38 takes the zero-vector convention of atan2(0, 0)), so
// no subnormal reaches these.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float div_ftz(float a, float b) {
  float r;
  asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
constexpr float kFltMin = 1.17549435e-38f;

// sqrt(x) for x >= 0 through the hardware reciprocal square root.
__device__ __forceinline__ float fast_sqrt(float x) { return x >= kFltMin ? x * rsqrt_ftz(x) : 0.f; }

// Packed float32 pairs (two independent fma.rn per instruction on sm_100+).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// W[t] . a, Wd[t] . a, Wdd[t] . a for both axes, with coefficient pairs
// (k, k+1) in packed registers: `row` holds the three zero-padded basis rows
// of timestep t, xv / yv the padded coefficient pairs.
template <int NC>
__device__ __forceinline__ void kin(const float* __restrict__ row,
                                    const float2 (&xv)[basis32_ncp(NC) / 2],
                                    const float2 (&yv)[basis32_ncp(NC) / 2], float (&o)[6]) {
  constexpr int NCP = basis32_ncp(NC);
#pragma unroll
  for (int mat = 0; mat < 3; ++mat) {
    float2 ax = f2(0.f, 0.f), ay = f2(0.f, 0.f);
#pragma unroll
    for (int k4 = 0; k4 < NCP; k4 += 4) {
      const float4 w = *reinterpret_cast<const float4*>(row + mat * NCP + k4);
      const float2 w01 = f2(w.x, w.y), w23 = f2(w.z, w.w);
      ax = fma2(w01, xv[k4 / 2], ax);
      ay = fma2(w01, yv[k4 / 2], ay);
      ax = fma2(w23, xv[k4 / 2 + 1], ax);
      ay = fma2(w23, yv[k4 / 2 + 1], ay);
    }
    o[2 * mat] = ax.x + ax.y;
    o[2 * mat + 1] = ay.x + ay.y;
  }
}

// Sum over the warp of the 2 n partial sums of the transposed contraction:
// on return lane (axis * 16 + k) holds the total of coefficient k of `axis`
// (recursive halving: at offset o a lane keeps the half of the slots selected
// by bit o of its index and adds its partner's copy of that half).
template <int NC, int NP>
__device__ __forceinline__ float warp_reduce_slots(const float2 (&wx)[NP], const float2 (&wy)[NP],
                                                   int lane) {
  float v[16];
  const bool hi = (lane & 16) != 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i < NC) {
      const float xv = (i & 1) ? wx[i / 2].y : wx[i / 2].x;
      const float yv = (i & 1) ? wy[i / 2].y : wy[i / 2].x;
      v[i] = (hi ? yv : xv) + __shfl_xor_sync(kFull, hi ? xv : yv, 16);
    } else {
      v[i] = 0.f;
    }
  }
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i)
      v[i] = (up ? v[i + o] : v[i]) + __shfl_xor_sync(kFull, up ? v[i] : v[i + o], o);
  }
  return v[0];
}

// Barrier of the warps that share one sample: named barrier 1 + grp for
// sample group grp < 4 of the CTA (constant ids: a run-time id would make the
// compiler reserve all 16 barriers per CTA).
__device__ __forceinline__ void group_barrier(int grp, int nthreads) {
  switch (grp) {
    case 0: asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory"); break;
    case 1: asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory"); break;
    case 2: asm volatile("bar.sync 3, %0;" ::"r"(nthreads) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(nthreads) : "memory"); break;
  }
}

// One sample per group of WPS warps (32 WPS lanes); a CTA holds blockDim.x /
// (32 WPS) groups (up to 4 with two warps per sample, one with four).  Larger
// CTAs share one staged copy of the basis among more samples.  Timestep t = s * 32 WPS +
// (warp-in-group) * 32 + lane for slot s; lanes with t >= m read a zero basis
// row, sit far from every obstacle and contribute nothing.
template <int NC, int SLOTS, int WPS, bool ROAD>
struct RegCap {
  // registers per thread: one timestep slot per 32 lanes needs about 70, the
  // rest is per-sample state; capped so that enough warps stay resident.  At
  // 4 warps per sample, 72 registers let 7 CTAs of 128 threads share an SM
  // (7 x 128 x 72 <= 65536), so 1000 samples fit one wave on 152 SMs; n = 16
  // needs 88 to avoid spills
  static constexpr int value =
      SLOTS * WPS >= 8 ? 255
                       : (SLOTS >= 4 ? 224
                                     : (SLOTS == 2 ? 144 : (WPS == 4 ? (NC <= 11 ? 72 : 88) : 96)));
};

// Rows 0..m-1 of the basis, then one zero row that lanes past the horizon
// read: their kinematics are zero and their residual rows contribute nothing.
// Threads first, first + step, ... copy.
template <int NC>
__device__ __forceinline__ void stage_basis(const Consts& c, int m, float* sW, int first, int step) {
  constexpr int ST = basis32_stride(NC);
  const float4* src = reinterpret_cast<const float4*>(c.basis32);
  float4* dst = reinterpret_cast<float4*>(sW);
  for (int i = first; i < (m + 1) * ST / 4; i += step)
    dst[i] = i < m * ST / 4 ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The scene's data in shared memory: the scaled obstacle trajectories
// ([N][4] float4) and the rows of M for N obstacles ([2][NC][NC]).
template <int NC>
__device__ __forceinline__ void stage_scene(const DevScene& sc, const double* __restrict__ obs,
                                            const Consts& c, const Params& prm, float4* sObs,
                                            float* sM, int first, int step) {
  const int N = sc.n_obs;
  for (int i = first; i < N; i += step) {
    // scaled trajectory: (x - x_o(t)) / a = x / a + (-x0/a) + (-vx dt / a) t,
    // constants duplicated for packed pairs of timesteps
    const double* o = obs + size_t(sc.obs_off + i) * 6;
    const double ia = 1.0 / o[4], ib = 1.0 / o[5];
    const float nx0 = float(-o[0] * ia), nvx = float(-o[2] * ia * prm.dt);
    const float ny0 = float(-o[1] * ib), nvy = float(-o[3] * ib * prm.dt);
    sObs[4 * i + 0] = make_float4(nx0, nx0, nvx, nvx);
    sObs[4 * i + 1] = make_float4(ny0, ny0, nvy, nvy);
    sObs[4 * i + 2] = make_float4(float(ia), float(ia), float(ib), float(ib));
    sObs[4 * i + 3] = make_float4(float(o[4]), float(o[5]), 0.f, 0.f);
  }
  for (int e = first; e < 2 * NC * NC; e += step) {
    const int ax_ = e / (NC * NC), k_ = (e / NC) % NC, i_ = e % NC;
    sM[e] = c.pj32[size_t((N * 2 + ax_) * NC + k_) * (2 * NC + c.ne) + i_];
  }
}

// Floats per sample group of the reduction table: one warp transposes through
// a [2n][RS] table (RS = 32 WPS + 4); with several warps each warp reduces with
// shuffles and the warps add their [32] results through a double-buffered
// [2][WPS][32] table.
template <int NC, int WPS>
__host__ __device__ constexpr int red_floats() {
  return WPS > 1 ? 2 * WPS * 32 : 2 * NC * (32 * WPS + 4);
}

// Step 1, the K iterations of Alg. 2 and the scoring of sample j by the
// calling warp's sample group (group = warp / WPS of the CTA).  sW: the basis
// rows; sObs, sM: the sample's scene data; sBuf ([warps][64]), sRedAll
// ([groups][red_floats]), sScore ([groups][WPS][2]) and sRef
// ([warps][6][SLOTS][32]) are the CTA's work areas; thr holds the calling
// warp's obstacle re-test levels (n_obs floats).
template <int NC, int SLOTS, int WPS, bool ROAD>
__device__ __forceinline__ void solve_sample(
    const DevScene& sc, int j, const float* sW, const float4* sObs, const float* sM, float* sBuf,
    float* sRedAll, float* sScore, float* sRef, float* thr, const double* __restrict__ pin,
    const Consts& c, const Params& prm, double* __restrict__ xi_out, double* __restrict__ r_out,
    double* __restrict__ cu_out, int* __restrict__ st_out) {
  constexpr int NCP = basis32_ncp(NC);
  constexpr int NP = NCP / 2;              // coefficient pairs
  constexpr int ST = basis32_stride(NC);
  constexpr int LPS = 32 * WPS;
  constexpr bool kPairSlots = SLOTS % 2 == 0;
  constexpr int RS = 32 * WPS + 4;         // row stride of the reduction table
  constexpr int RED = red_floats<NC, WPS>();
  const int m = prm.m;
  const int ns = prm.n_seg;
  const int N = sc.n_obs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / WPS, wig = warp % WPS;
  const int gl = wig * 32 + lane;                           // lane within the sample group
  float* xbuf = sBuf + warp * 64;      // slot layout: xi_bar, then delta (per warp copy)
  float* vbuf = xbuf + 32;             // slot layout: lambda + rho w - delta
  float* sRed = sRedAll + grp * RED;
  float* ref = sRef + warp * 6 * SLOTS * 32 + lane;   // ref[(q * SLOTS + s) * 32]
  // Obstacle i can hold a point of this warp's timesteps only once the
  // trajectory has moved by (scaled) thr[i] - moved - 1 since it was last
  // tested: positions are convex combinations of the coefficients (Bernstein
  // rows are nonnegative and sum to one), so no point moves further than the
  // largest coefficient change.  Skipped obstacles contribute exactly zero.
  for (int i = lane; i < N; i += 32) thr[i] = -3.0e38f;
  float ia_max = 0.f, ib_max = 0.f;
  for (int i = lane; i < N; i += 32) {
    ia_max = fmaxf(ia_max, sObs[4 * i + 2].x);
    ib_max = fmaxf(ib_max, sObs[4 * i + 2].z);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    ia_max = fmaxf(ia_max, __shfl_xor_sync(kFull, ia_max, o));
    ib_max = fmaxf(ib_max, __shfl_xor_sync(kFull, ib_max, o));
  }
  float moved = 0.f;   // bound on the scaled movement of any point since iteration 0
  // warp maximum of the last xi-step's scaled movement; it is added to `moved`
  // just before the next obstacle test, so the reduction's latency overlaps the
  // kinematics of the next iteration
  float moved_step = 0.f;

  // ---- per-lane coefficient slot: Step 1 and the row of M
  const int axis = lane >> 4, kk = lane & 15;
  const bool valid = kk < NC;
  const float* Mrow_s = sM + (axis * NC + (valid ? kk : 0)) * NC;
  // shapes with few timestep slots keep the reference kinematics and the row of
  // M in registers; the others read them from shared memory
  constexpr bool kRegState = WPS == 1 && SLOTS <= 4;
  constexpr bool kRegM = kRegState || (WPS == 2 && SLOTS <= 2);
  float Mrow_r[kRegM ? NC : 1];
#pragma unroll
  for (int i = 0; i < (kRegM ? NC : 1); ++i) Mrow_r[i] = Mrow_s[i];
  float xb_l = 0.f;     // xi_bar of this lane's slot
  pdl_wait();           // p comes from the sampling kernel
  if (valid) {
    // xi_bar = Gs p_axis + Hs b_axis (x uses the v_d entries, y the y_d entries),
    // applied in float64: at high polynomial degree the Step-1 map has entries
    // of order 1e3 whose products cancel to the coefficients' size.  With goal
    // entries b_axis also holds x_f (x) or y_f (y); the final ydot = 0 adds nothing.
    const double* s1 = c.s1_64 + size_t(axis * NC + kk) * (ns + c.ne);
    const double* pj = pin + size_t(j) * prm.d_p;
    double xb = 0.0;
    for (int q = 0; q < ns; ++q) xb = fma(s1[q], pj[(axis == 0 ? ns : 0) + q], xb);
    xb = fma(s1[ns], sc.ego[axis], xb);
    xb = fma(s1[ns + 1], sc.ego[axis + 2], xb);
    xb = fma(s1[ns + 2], sc.ego[axis + 4], xb);
    if (prm.goal) xb = fma(s1[ns + 3], pj[2 * ns + axis], xb);
    xb_l = float(xb);
  }
  xbuf[lane] = xb_l;     // padding slots hold 0: they meet zero basis columns
  __syncwarp();

  int tcl[SLOTS];     // basis row: t, or the zero row m for t >= m
  float act[SLOTS];   // 1 for t < m, else 0
  float tt[SLOTS];    // timestep index as float (obstacle tables hold per-step rates)
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int t = s * LPS + gl;
    tcl[s] = min(t, m);
    act[s] = t < m ? 1.f : 0.f;
    tt[s] = float(t);
  }

  auto load_iterate = [&](float2 (&xv)[NP], float2 (&yv)[NP]) {
#pragma unroll
    for (int i4 = 0; i4 < NCP; i4 += 4) {
      const float4 a = *reinterpret_cast<const float4*>(xbuf + i4);
      const float4 b = *reinterpret_cast<const float4*>(xbuf + 16 + i4);
      xv[i4 / 2] = f2(a.x, a.y); xv[i4 / 2 + 1] = f2(a.z, a.w);
      yv[i4 / 2] = f2(b.x, b.y); yv[i4 / 2 + 1] = f2(b.z, b.w);
    }
  };

  float rref[kRegState ? SLOTS : 1][6];   // reference kinematics at xi_bar (register copy)
  // ---- reference kinematics at xi_bar
  {
    float2 xv[NP], yv[NP];
    load_iterate(xv, yv);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      float o[6];
      kin<NC>(sW + tcl[s] * ST, xv, yv, o);
      // a lane past the horizon is placed 10^15 m down the road: every obstacle
      // test sees it outside (its scaled squared distance stays finite, far
      // above 1), so the tests need no per-slot mask.  Its other kinematics
      // and residual rows stay zero.
      if (act[s] == 0.f) o[0] = 1.0e15f;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        if constexpr (kRegState) rref[s][q] = o[q];
        else ref[(q * SLOTS + s) * 32] = o[q];
      }
    }
  }
  __syncwarp();
  xbuf[lane] = 0.f;    // delta^0 = 0

  const float rho = float(prm.rho);
  const float hrho = 0.5f * rho;
  const float v_min = float(prm.v_min), v_max = float(prm.v_max), a_max = float(prm.a_max);
  const float kmax = float(prm.kappa_max), inv_kmax = float(1.0 / prm.kappa_max);
  const float c_max = float(prm.c_max);
  const float kr = float(fabs(sc.kappa_road));
  const float y_lb = float(sc.y_lb), y_ub = float(sc.y_ub);

  float da[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) da[s] = 0.f;
  // road profile: curvature at the previous iterate (Eq. clip_d_v), lane limits
  // at the current one; without a profile both are the scene's constants
  constexpr bool road = ROAD;
  float xprev[SLOTS];

  float lam = 0.f, dl = 0.f;     // lambda and delta of this lane's slot
  float r_acc = 0.f, cu_acc = 0.f;

  for (int it = 0;; ++it) {
    __syncwarp();
    float2 xv[NP], yv[NP];
    load_iterate(xv, yv);

    // ---- A: kinematics at the lane's timesteps
    float px[SLOTS], py[SLOTS], vx[SLOTS], vy[SLOTS], ax[SLOTS], ay[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      float o[6], r6[6];
      kin<NC>(sW + tcl[s] * ST, xv, yv, o);
#pragma unroll
      for (int q = 0; q < 6; ++q) r6[q] = kRegState ? rref[s][q] : ref[(q * SLOTS + s) * 32];
      px[s] = r6[0] + o[0]; py[s] = r6[1] + o[1];
      vx[s] = r6[2] + o[2]; vy[s] = r6[3] + o[3];
      ax[s] = r6[4] + o[4]; ay[s] = r6[5] + o[5];
    }

    if (it == prm.K) {
      // ---- scoring of xi^K (Alg. 1 line 9 and the Sec. V-A cost)
      float coll[SLOTS];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) coll[s] = 0.f;
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        const float4 q0 = sObs[4 * i], q1 = sObs[4 * i + 1], q2 = sObs[4 * i + 2];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const float sx = fmaf(px[s], q2.x, fmaf(q0.z, tt[s], q0.x));
          const float sy = fmaf(py[s], q2.z, fmaf(q1.z, tt[s], q1.x));
          coll[s] += fmaxf(0.f, 1.f - fmaf(sx, sx, sy * sy));
        }
      }
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const float sp = fast_sqrt(fmaf(vx[s], vx[s], vy[s] * vy[s]));
        const float am = fast_sqrt(fmaf(ax[s], ax[s], ay[s] * ay[s]));
        const float kap =
            sp > 0.f ? __fdividef(fmaf(ay[s], vx[s], -(ax[s] * vy[s])), sp * sp * sp) : 0.f;
        float kro = kr, ylo = y_lb, yup = y_ub;
        if (road) {
          road_eval<float>(sc, px[s], &kro, &ylo, &yup);
          kro = fabsf(kro);
        }
        const float rt = coll[s] + fmaxf(0.f, sp - v_max) + fmaxf(0.f, am - a_max) +
                         fmaxf(0.f, fabsf(kap) - kmax) +
                         fmaxf(0.f, fmaf(vx[s] * vx[s], kro, -c_max)) +
                         fmaxf(0.f, py[s] - yup) + fmaxf(0.f, ylo - py[s]);
        const float dv = sp - v_max;
        r_acc = fmaf(act[s], rt, r_acc);
        cu_acc = fmaf(act[s] * dv, dv, cu_acc);
      }
      break;
    }

    moved = fmaf(1.41422f, moved_step, moved);
    // ---- B: obstacle projection, accumulated residual sum_i (h_o,i - p).
    // For every obstacle within reach, one pass computes the scaled offsets of
    // all slots and gives the points inside its ellipse (d < 1) the correction
    // (x - x_o, y - y_o)(1/d - 1).  An obstacle that holds a point stays within
    // reach for the next iteration whatever its exact level (min d < 1), so it
    // is re-armed without a warp reduction; otherwise its skip level is
    // re-armed from the warp minimum of the scaled distance.  Either way the
    // next iteration tests the same obstacles.
    float ex[SLOTS], ey[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) { ex[s] = 0.f; ey[s] = 0.f; }
    for (int i0 = 0; i0 < N; i0 += 32) {
      const int nc = min(32, N - i0);
      // obstacles that may be within reach (warp-uniform mask)
      unsigned near = __ballot_sync(kFull, lane < nc && thr[i0 + lane] - moved <= 1.001f);
      while (near) {
        const int ii = __ffs(near) - 1;
        near &= near - 1u;
        const float4 q0 = sObs[4 * (i0 + ii)], q1 = sObs[4 * (i0 + ii) + 1];
        const float4 q2 = sObs[4 * (i0 + ii) + 2], q3 = sObs[4 * (i0 + ii) + 3];
        float sxs[SLOTS], sys[SLOTS], d2s[SLOTS];
        float dmin = 3.0e38f;
        bool in_any = false;
        if constexpr (kPairSlots) {
#pragma unroll
          for (int s = 0; s < SLOTS; s += 2) {
            const float2 tp = f2(tt[s], tt[s + 1]);
            const float2 sx = fma2(f2(px[s], px[s + 1]), f2(q2.x, q2.y),
                                   fma2(f2(q0.z, q0.w), tp, f2(q0.x, q0.y)));
            const float2 sy = fma2(f2(py[s], py[s + 1]), f2(q2.z, q2.w),
                                   fma2(f2(q1.z, q1.w), tp, f2(q1.x, q1.y)));
            const float2 d2 = fma2(sx, sx, mul2(sy, sy));
            sxs[s] = sx.x; sxs[s + 1] = sx.y;
            sys[s] = sy.x; sys[s + 1] = sy.y;
            d2s[s] = d2.x; d2s[s + 1] = d2.y;
          }
        } else {
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) {
            sxs[s] = fmaf(px[s], q2.x, fmaf(q0.z, tt[s], q0.x));
            sys[s] = fmaf(py[s], q2.z, fmaf(q1.z, tt[s], q1.x));
            d2s[s] = fmaf(sxs[s], sxs[s], sys[s] * sys[s]);
          }
        }
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          dmin = fminf(dmin, d2s[s]);
          in_any |= d2s[s] < 1.f;
        }
        if (__any_sync(kFull, in_any)) {
          if (lane == 0) thr[i0 + ii] = -3.0e38f;
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) {
            // inside (d < 1): scale the offset onto the ellipse; at the centre
            // atan2(0, 0) = 0 gives h = (x_o + a, y_o); outside: no change
            const bool in = d2s[s] < 1.f;
            const bool pos = d2s[s] >= kFltMin;
            const float rs = rsqrt_ftz(d2s[s]);
            const float g = (in && pos) ? rs - 1.f : 0.f;
            ex[s] = fmaf(g * q3.x, sxs[s], ex[s]) + ((in && !pos) ? q3.x : 0.f);
            ey[s] = fmaf(g * q3.y, sys[s], ey[s]);
          }
        } else {
          // warp minimum of a nonnegative float: integer order of its bits
          dmin = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(dmin)));
          if (lane == 0) thr[i0 + ii] = fast_sqrt(dmin) + moved;
        }
      }
    }

    // ---- C: velocity / acceleration / lane rows and the transposed contraction
    float2 wx[NP], wy[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) { wx[k] = f2(0.f, 0.f); wy[k] = f2(0.f, 0.f); }
    bool wany = false;     // some slot of this warp has a nonzero row (warp-uniform)
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const float v2 = fmaf(vx[s], vx[s], vy[s] * vy[s]);
      const bool vp = v2 >= kFltMin;
      const float rv = rsqrt_ftz(v2);
      const float cv = vp ? vx[s] * rv : 1.f, sv = vp ? vy[s] * rv : 0.f, sp = vp ? v2 * rv : 0.f;
      const float a2 = fmaf(ax[s], ax[s], ay[s] * ay[s]);
      const bool ap = a2 >= kFltMin;
      const float ra = rsqrt_ftz(a2);
      const float ca = ap ? ax[s] * ra : 1.f, sa = ap ? ay[s] * ra : 0.f, am = ap ? a2 * ra : 0.f;
      const float S = fabsf(fmaf(sa, cv, -(ca * sv)));       // |sin(alpha_a - alpha_v)|
      const float dap = (it == 0) ? fminf(am, a_max) : da[s];
      const float vmin_b = fmaxf(v_min, fast_sqrt(dap * S * inv_kmax));
      float vmax_b = v_max;
      float krs = kr, ylbs = y_lb, yubs = y_ub;
      if (road) {
        float unused;
        road_eval<float>(sc, it == 0 ? px[s] : xprev[s], &krs, &unused, &unused);
        krs = fabsf(krs);
        road_eval<float>(sc, px[s], &unused, &ylbs, &yubs);
        xprev[s] = px[s];
      }
      if (krs > 0.f) {
        const float tc = krs * cv * cv;
        if (tc >= kFltMin) vmax_b = fminf(v_max, fast_sqrt(div_ftz(c_max, tc)));
      }
      const float dv = fminf(fmaxf(sp, vmin_b), vmax_b);
      const float kd = dv * dv * kmax;
      const float amax_b = (S * a_max <= kd) ? a_max : div_ftz(kd, S);
      const float dan = fminf(am, amax_b);
      da[s] = dan;
      // Unclipped, h_v = v and h_a = a exactly (d = |v|, |a| with the same
      // direction): their rows are zero, not the rounding noise of d (cos, sin) - v.
      // Lanes past the horizon meet the zero basis row in the contraction.
      const bool vclip = dv != sp, aclip = dan != am;
      const float evx = vclip ? fmaf(dv, cv, -vx[s]) : 0.f;
      const float evy = vclip ? fmaf(dv, sv, -vy[s]) : 0.f;
      const float eax = aclip ? fmaf(dan, ca, -ax[s]) : 0.f;
      const float eay = aclip ? fmaf(dan, sa, -ay[s]) : 0.f;
      const float ely = fminf(fmaxf(py[s], ylbs), yubs) - py[s];
      const float exs = ex[s];
      const float eoy = ey[s] + ely;
      // a slot whose rows are zero on every lane adds nothing to the
      // transposed contraction (all its constraints hold): skip it
      const bool nz = act[s] > 0.f && (vclip | aclip | (exs != 0.f) | (eoy != 0.f));
      if (__any_sync(kFull, nz)) {
        wany = true;
        const float* row = sW + tcl[s] * ST;
        const float2 ex_[3] = {f2(exs, exs), f2(evx, evx), f2(eax, eax)};
        const float2 ey_[3] = {f2(eoy, eoy), f2(evy, evy), f2(eay, eay)};
#pragma unroll
        for (int mat = 0; mat < 3; ++mat) {
#pragma unroll
          for (int k4 = 0; k4 < NCP; k4 += 4) {
            const float4 w = *reinterpret_cast<const float4*>(row + mat * NCP + k4);
            const float2 w01 = f2(w.x, w.y), w23 = f2(w.z, w.w);
            wx[k4 / 2] = fma2(w01, ex_[mat], wx[k4 / 2]);
            wy[k4 / 2] = fma2(w01, ey_[mat], wy[k4 / 2]);
            wx[k4 / 2 + 1] = fma2(w23, ex_[mat], wx[k4 / 2 + 1]);
            wy[k4 / 2 + 1] = fma2(w23, ey_[mat], wy[k4 / 2 + 1]);
          }
        }
      }
    }

    // ---- D: reduce over the sample's lanes through a shared-memory transpose,
    // multipliers, xi-step in increment form
    float wl;
    if constexpr (WPS > 1) {
      // a warp whose slots were all skipped has all-zero partial sums
      const float part = wany ? warp_reduce_slots<NC, NP>(wx, wy, lane) : 0.f;
      float* rt = sRed + (it & 1) * WPS * 32;
      rt[wig * 32 + lane] = part;
      group_barrier(grp, LPS);
      wl = 0.f;
#pragma unroll
      for (int w = 0; w < WPS; ++w) wl += rt[w * 32 + lane];
    } else {
      float* rt = sRed;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        rt[k * RS + gl] = (k & 1) ? wx[k / 2].y : wx[k / 2].x;
        rt[(NC + k) * RS + gl] = (k & 1) ? wy[k / 2].y : wy[k / 2].x;
      }
      __syncwarp();
      wl = 0.f;
      if (valid) {
        const float4* rrow = reinterpret_cast<const float4*>(rt + (axis * NC + kk) * RS);
        const float4 a = rrow[0];
        float2 lo = f2(a.x, a.y), hi = f2(a.z, a.w);
#pragma unroll
        for (int c4 = 1; c4 < 8 * WPS; ++c4) {
          const float4 b = rrow[c4];
          lo = add2(lo, f2(b.x, b.y));
          hi = add2(hi, f2(b.z, b.w));
        }
        wl = (lo.x + lo.y) + (hi.x + hi.y);
      }
    }
    if (valid) {
      if (it > 0) lam = fmaf(hrho, wl, lam);
      vbuf[lane] = fmaf(rho, wl, lam) - dl;
    }
    __syncwarp();
    float acc_step = 0.f;
    if (valid) {
      // this axis's half of the vector, 16-byte aligned (entries NC..15 unused)
      const float4* vb4 = reinterpret_cast<const float4*>(vbuf + axis * 16);
      float vb[NCP];
#pragma unroll
      for (int i4 = 0; i4 < NCP / 4; ++i4) {
        const float4 v = vb4[i4];
        vb[4 * i4] = v.x; vb[4 * i4 + 1] = v.y; vb[4 * i4 + 2] = v.z; vb[4 * i4 + 3] = v.w;
      }
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int i = 0; i < NC; i += 2) {
        acc0 = fmaf(kRegM ? Mrow_r[i] : Mrow_s[i], vb[i], acc0);
        if (i + 1 < NC) acc1 = fmaf(kRegM ? Mrow_r[i + 1] : Mrow_s[i + 1], vb[i + 1], acc1);
      }
      acc_step = acc0 + acc1;
      dl += acc_step;
      xbuf[lane] = dl;
    }
    {
      // scaled bound on how far any point moves in this step
      const float mv = valid ? fabsf(acc_step) * (axis ? ib_max : ia_max) : 0.f;
      moved_step = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(mv)));
    }
  }

  // ---- outputs
  pdl_trigger();
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    r_acc += __shfl_xor_sync(kFull, r_acc, o);
    cu_acc += __shfl_xor_sync(kFull, cu_acc, o);
  }
  if constexpr (WPS > 1) {
    float* sc2 = sScore + grp * WPS * 2;
    if (lane == 0) { sc2[2 * wig] = r_acc; sc2[2 * wig + 1] = cu_acc; }
    group_barrier(grp, LPS);
    r_acc = 0.f;
    cu_acc = 0.f;
#pragma unroll
    for (int w = 0; w < WPS; ++w) { r_acc += sc2[2 * w]; cu_acc += sc2[2 * w + 1]; }
  }
  if (wig == 0) {
    if (st_out != nullptr) {
      // per-sample status: the solution, its residual and its cost are finite
      const bool bad_xi = __any_sync(kFull, valid && !(isfinite(xb_l) && isfinite(dl)));
      if (lane == 0)
        st_out[j] = (bad_xi || !isfinite(r_acc) || !isfinite(cu_acc)) ? PLAN_ENONFINITE : PLAN_OK;
    }
    if (lane == 0) {
      r_out[j] = double(r_acc);
      cu_out[j] = double(cu_acc);
    }
    if (xi_out != nullptr && valid)
      xi_out[size_t(j) * 2 * NC + axis * NC + kk] = double(xb_l) + double(dl);
  }
}

// One tile (up to samples_per_cta samples of one scene) per CTA.
template <int NC, int SLOTS, int WPS, bool ROAD>
__global__ void __launch_bounds__(256) __maxnreg__((RegCap<NC, SLOTS, WPS, ROAD>::value))
fused_kernel(const DevScene* __restrict__ scenes, const Layout* __restrict__ layout,
             const double* __restrict__ obs, const Tile* __restrict__ tiles,
             const double* __restrict__ pin, Consts c, Params prm,
             double* __restrict__ xi_out, double* __restrict__ r_out,
             double* __restrict__ cu_out, int* __restrict__ st_out) {
  constexpr int ST = basis32_stride(NC);
  constexpr int RED = red_floats<NC, WPS>();
  extern __shared__ __align__(16) float smem[];
  const int m = prm.m;
  const Tile tile = tiles[blockIdx.x];
  const DevScene& sc = scenes[tile.scene];
  const int N = sc.n_obs;
  const int warps = blockDim.x >> 5;
  const int groups = warps / WPS;

  float* sW = smem;                                          // [m + 1][ST]
  float4* sObs = reinterpret_cast<float4*>(smem + (m + 1) * ST);   // [N][4]
  float* sBuf = reinterpret_cast<float*>(sObs + 4 * N);      // [warps][64]
  float* sRedAll = sBuf + 64 * warps;                        // [groups][RED]
  float* sScore = sRedAll + groups * RED;                    // [groups][WPS][2]
  float* sM = sScore + groups * WPS * 2;                     // [2][NC][NC] rows of M
  float* sRef = sM + 2 * NC * NC;                            // [warps][6][SLOTS][32]
  float* sThr = sRef + warps * 6 * SLOTS * 32;               // [warps][N] obstacle re-test levels

  stage_basis<NC>(c, m, sW, threadIdx.x, blockDim.x);
  stage_scene<NC>(sc, obs, c, prm, sObs, sM, threadIdx.x, blockDim.x);
  __syncthreads();

  const int warp = threadIdx.x >> 5;
  const int grp = warp / WPS;
  if (grp >= tile.count) return;
  solve_sample<NC, SLOTS, WPS, ROAD>(sc, layout[tile.scene].off + tile.first + grp, sW, sObs, sM,
                                     sBuf, sRedAll, sScore, sRef, sThr + warp * N, pin, c, prm,
                                     xi_out, r_out, cu_out, st_out);
}

// The persistent form exists for the shapes with four or more timestep slots
// per lane: one warp per sample, and two warps per sample beyond 128 steps
// (the shapes chosen for launches of more than one wave); the others always
// launch one tile per CTA.  Its registers: the sample loop keeps a few more
// values live than one tile does; where the one-tile form is uncapped, 168 keep
// three CTAs of 128 threads per SM (3 x 128 x 168 <= 65536).
template <int SLOTS>
constexpr bool has_persistent() { return SLOTS >= 4; }

template <int NC, int SLOTS, int WPS, bool ROAD>
struct RegCapPersistent {
  static constexpr int value = SLOTS * WPS >= 8 ? 168 : RegCap<NC, SLOTS, WPS, ROAD>::value;
};

// Persistent form, for launches of more than one wave of CTAs: the grid is one
// wave, each CTA stages the basis once, and each sample group takes the next
// sample (a global index into p) from the counter work[0] until none is left,
// so a group whose sample finished early starts another one instead of
// waiting for the other groups of its CTA.  Each group keeps its own copy of
// its sample's scene data (obstacles and rows of M, for up to max_obs
// obstacles) and restages it when the next sample belongs to another scene.
// work[1] counts the groups that found no sample left; the last of them resets
// both counters to zero for the next launch.  No thread waits on another CTA.
template <int NC, int SLOTS, int WPS, bool ROAD>
__global__ void __launch_bounds__(256) __maxnreg__((RegCapPersistent<NC, SLOTS, WPS, ROAD>::value))
fused_persistent_kernel(const DevScene* __restrict__ scenes, const double* __restrict__ obs,
                        const int* __restrict__ sample_scene, int total, int* work,
                        const double* __restrict__ pin, Consts c, Params prm,
                        double* __restrict__ xi_out, double* __restrict__ r_out,
                        double* __restrict__ cu_out, int* __restrict__ st_out) {
  constexpr int ST = basis32_stride(NC);
  constexpr int LPS = 32 * WPS;
  constexpr int RED = red_floats<NC, WPS>();
  extern __shared__ __align__(16) float smem[];
  const int m = prm.m;
  const int NO = prm.max_obs;
  const int warps = blockDim.x >> 5;
  const int groups = warps / WPS;

  float* sW = smem;                                                   // [m + 1][ST]
  float4* sObsAll = reinterpret_cast<float4*>(smem + (m + 1) * ST);   // [groups][NO][4]
  float* sBuf = reinterpret_cast<float*>(sObsAll + 4 * NO * groups);  // [warps][64]
  float* sRedAll = sBuf + 64 * warps;                                 // [groups][RED]
  float* sScore = sRedAll + groups * RED;                             // [groups][WPS][2]
  float* sMAll = sScore + groups * WPS * 2;                           // [groups][2][NC][NC]
  float* sRef = sMAll + groups * 2 * NC * NC;                         // [warps][6][SLOTS][32]
  float* sThr = sRef + warps * 6 * SLOTS * 32;                        // [warps][NO]
  int* sTicket = reinterpret_cast<int*>(sThr + warps * NO);           // [groups]

  stage_basis<NC>(c, m, sW, threadIdx.x, blockDim.x);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / WPS, wig = warp % WPS;
  const int gl = wig * 32 + lane;
  float4* sObs = sObsAll + 4 * NO * grp;
  float* sM = sMAll + grp * 2 * NC * NC;
  // the previous launch on the stream resets the counters as it ends, and a
  // programmatic launch may start before that: take no sample until it is done
  pdl_wait();
  int cur = -1;
  for (;;) {
    int j;
    if constexpr (WPS == 1) {
      int t = 0;
      if (lane == 0) t = atomicAdd(work, 1);
      j = __shfl_sync(kFull, t, 0);
    } else {
      // every warp of the group has read the previous ticket: it passed the
      // group barriers of that sample's solve since
      if (gl == 0) sTicket[grp] = atomicAdd(work, 1);
      group_barrier(grp, LPS);
      j = sTicket[grp];
    }
    if (j >= total) break;
    const int s = sample_scene[j];
    if (s != cur) {
      // the group's warps are past the previous sample: restage its scene data
      stage_scene<NC>(scenes[s], obs, c, prm, sObs, sM, gl, LPS);
      if constexpr (WPS == 1) __syncwarp(); else group_barrier(grp, LPS);
      cur = s;
    }
    solve_sample<NC, SLOTS, WPS, ROAD>(scenes[s], j, sW, sObs, sM, sBuf, sRedAll, sScore, sRef,
                                       sThr + warp * NO, pin, c, prm, xi_out, r_out, cu_out,
                                       st_out);
  }
  if (gl == 0) {
    __threadfence();   // this group's last ticket is taken before it counts itself done
    if (atomicAdd(work + 1, 1) == int(gridDim.x) * groups - 1) {
      atomicExch(work, 0);
      atomicExch(work + 1, 0);
    }
  }
}

template <int NC, int SLOTS, int WPS>
size_t smem_bytes(const Params& prm, int spc) {
  const int warps = spc * WPS;
  const int red = red_floats<NC, WPS>();
  size_t f = size_t(prm.m + 1) * basis32_stride(NC) + 16 * prm.max_obs + 64 * warps + spc * red +
             spc * WPS * 2 + 2 * NC * NC + size_t(6) * SLOTS * 32 * warps + size_t(warps) * prm.max_obs;
  return f * sizeof(float);
}

// Shared memory of fused_persistent_kernel: the basis once, the scene data and
// the reduction table per group, the work areas per warp, one ticket per group.
template <int NC, int SLOTS, int WPS>
size_t smem_bytes_persistent(const Params& prm, int spc) {
  const int warps = spc * WPS;
  const size_t per_group =
      size_t(16) * prm.max_obs + 2 * NC * NC + red_floats<NC, WPS>() + WPS * 2 + 1;
  const size_t per_warp = 64 + size_t(6) * SLOTS * 32 + prm.max_obs;
  const size_t f = size_t(prm.m + 1) * basis32_stride(NC) + spc * per_group + warps * per_warp;
  return f * sizeof(float);
}

// Resident CTAs per SM of a kernel at a block size and dynamic shared memory,
// from the occupancy calculator, cached per (device, kernel, block, bytes).
inline cudaError_t blocks_per_sm(const void* fn, int threads, size_t smem, int* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(dev, fn, threads, smem);
  std::lock_guard<std::mutex> lk(mu);
  const auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  int n = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
  if (e != cudaSuccess) return e;
  if (n < 1) return cudaErrorInvalidConfiguration;
  cache[key] = n;
  *out = n;
  return cudaSuccess;
}

template <int NC, int SLOTS, int WPS, bool ROAD>
cudaError_t launch_t(const FusedLaunch& L, const Consts& c, const Params& prm, cudaStream_t s) {
  const int threads = L.spc * WPS * 32;
  bool persist = has_persistent<SLOTS>() && L.persist == PLAN_PERSIST_ON;
  if (has_persistent<SLOTS>() && L.persist == PLAN_PERSIST_AUTO) {
    // persistent once the tiles need more than one wave of CTAs
    int per_sm = 0;
    const cudaError_t e =
        blocks_per_sm(reinterpret_cast<const void*>(fused_kernel<NC, SLOTS, WPS, ROAD>), threads,
                      smem_bytes<NC, SLOTS, WPS>(prm, L.spc), &per_sm);
    if (e != cudaSuccess) return e;
    persist = L.n_tiles > per_sm * L.sms;
  }
  if (!persist)
    return launch_pdl(fused_kernel<NC, SLOTS, WPS, ROAD>, dim3(L.n_tiles), dim3(threads),
                      smem_bytes<NC, SLOTS, WPS>(prm, L.spc), s, L.scenes, L.layout, L.obs, L.tiles,
                      L.p, c, prm, L.xi, L.r, L.cu, L.st);
  if constexpr (has_persistent<SLOTS>()) {
    auto* fn = fused_persistent_kernel<NC, SLOTS, WPS, ROAD>;
    const size_t bytes = smem_bytes_persistent<NC, SLOTS, WPS>(prm, L.spc);
    int per_sm = 0;
    const cudaError_t e = blocks_per_sm(reinterpret_cast<const void*>(fn), threads, bytes, &per_sm);
    if (e != cudaSuccess) return e;
    const int ctas = std::min(per_sm * L.sms, (L.total + L.spc - 1) / L.spc);
    return launch_pdl(fn, dim3(ctas), dim3(threads), bytes, s, L.scenes, L.obs, L.sample_scene,
                      L.total, L.work, L.p, c, prm, L.xi, L.r, L.cu, L.st);
  }
  return cudaErrorInvalidValue;   // not reached: persist is false without the form
}

template <int NC, int SLOTS, int WPS, bool ROAD>
void set_attr() {
  // every CTA stages the basis: ask for the largest shared-memory carveout so
  // that occupancy is bounded by registers, not by the L1 / shared split
  cudaFuncSetAttribute(fused_kernel<NC, SLOTS, WPS, ROAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       200 * 1024);
  cudaFuncSetAttribute(fused_kernel<NC, SLOTS, WPS, ROAD>,
                       cudaFuncAttributePreferredSharedMemoryCarveout,
                       int(cudaSharedmemCarveoutMaxShared));
  if constexpr (has_persistent<SLOTS>()) {
    cudaFuncSetAttribute(fused_persistent_kernel<NC, SLOTS, WPS, ROAD>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(fused_persistent_kernel<NC, SLOTS, WPS, ROAD>,
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
  }
}

template <int NC, bool ROAD>
void set_attr_nc() {
  set_attr<NC, 4, 1, ROAD>(); set_attr<NC, 8, 1, ROAD>();
  set_attr<NC, 2, 2, ROAD>(); set_attr<NC, 4, 2, ROAD>();
  set_attr<NC, 1, 4, ROAD>(); set_attr<NC, 2, 4, ROAD>();
}

template <int NC, bool ROAD>
cudaError_t launch_nc(const FusedLaunch& L, const Consts& c, const Params& prm, cudaStream_t s) {
  // timestep slots per lane: horizons up to 128 steps fit half as many
  const bool short_h = prm.m <= 128;
  if (L.wps == 1)
    return short_h ? launch_t<NC, 4, 1, ROAD>(L, c, prm, s) : launch_t<NC, 8, 1, ROAD>(L, c, prm, s);
  if (L.wps == 2)
    return short_h ? launch_t<NC, 2, 2, ROAD>(L, c, prm, s) : launch_t<NC, 4, 2, ROAD>(L, c, prm, s);
  if (L.wps == 4)
    return short_h ? launch_t<NC, 1, 4, ROAD>(L, c, prm, s) : launch_t<NC, 2, 4, ROAD>(L, c, prm, s);
  return cudaErrorInvalidValue;
}

template <bool ROAD>
cudaError_t launch_road(const FusedLaunch& L, const Consts& c, const Params& prm, cudaStream_t s) {
  if (prm.n == 8) return launch_nc<8, ROAD>(L, c, prm, s);
  if (prm.n == 11) return launch_nc<11, ROAD>(L, c, prm, s);
  if (prm.n == 16) return launch_nc<16, ROAD>(L, c, prm, s);
  return cudaErrorInvalidValue;
}

template <bool ROAD>
void setup_road() {
  set_attr_nc<8, ROAD>();
  set_attr_nc<11, ROAD>();
  set_attr_nc<16, ROAD>();
}

}  // namespace

// The road-profile instantiations live in k_fused_road.cu (compiled in parallel).
void fused_setup_road();
cudaError_t launch_fused_f32_road(const FusedLaunch& L, const Consts& c, const Params& prm,
                                  cudaStream_t s);

}  // namespace plan

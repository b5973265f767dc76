// Fused FP32 lower-level solve: Step 1 (Alg. 1 line 7 through the folded KKT
// inverse of Eq. over_3), all K iterations of Alg. 2 and the scoring of
// Alg. 1 line 9 / Sec. V-A, one warp per sample, all state on chip.
//
// Per iteration and sample the warp
//   A. evaluates x, y and their derivatives at the lane's timesteps
//      t = s*32 + lane (Eq. param; basis staged in shared memory),
//   B. projects onto every obstacle ellipse (Eqs. split_alpha_o, clip_d_o),
//   C. projects velocity and acceleration (Eqs. clip_d_v, clip_d_a), the lane
//      rows (Eq. update_slack) and accumulates the transposed contraction
//        w = F^T (h - F xi) + G^T (e - s - G xi),
//   D. reduce-scatters w over the warp, updates the multipliers
//      lambda += rho/2 w (Eq. update_lagrange) and takes the xi-step of
//      Eq. split_xy in folded form
//        xi' = (M xi_bar + C b0) + M (lambda + rho w) + (rho M P) xi,
//      which equals M (xi_bar + lambda + rho F^T h + rho G^T (e - s)) + C b0
//      because F^T h + G^T (e - s) = w + P xi with P = F^T F + G^T G.
//
// The closed form of Eq. split_alpha_o is used without trigonometry: for an
// obstacle with scaled offset (sx, sy) = ((x - x_o)/a, (y - y_o)/b) and
// d^2 = sx^2 + sy^2, cos(alpha) = sx/d, sin(alpha) = sy/d, so the clipped
// point h = o + (a max(1,d) cos, b max(1,d) sin) differs from the trajectory
// point by (x - x_o, y - y_o) (1/d - 1) when d < 1 and by zero otherwise.
#include "internal.cuh"

namespace plan {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int NC>
__device__ __forceinline__ float reduce_scatter(const float (&wx)[NC], const float (&wy)[NC],
                                                int lane) {
  // Logical slots: x coefficient k -> k, y coefficient k -> 16 + k.  After
  // five halving exchanges lane l holds the warp sum of slot l.
  float v[16];
  const bool up16 = lane & 16;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < NC) {
      float send = up16 ? wx[k] : wy[k];
      float keep = up16 ? wy[k] : wx[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, 16);
    } else {
      v[k] = 0.f;
    }
  }
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      float send = up ? v[k] : v[k + o];
      float keep = up ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

template <int NC, int SLOTS>
__global__ void __launch_bounds__(256)
fused_kernel(const DevScene* __restrict__ scenes, const Layout* __restrict__ layout,
             const double* __restrict__ obs, const Tile* __restrict__ tiles,
             const double* __restrict__ pin, Consts c, Params prm,
             double* __restrict__ xi_out, double* __restrict__ r_out,
             double* __restrict__ cu_out) {
  extern __shared__ __align__(16) float smem[];
  const int m = prm.m;
  const int ns = prm.n_seg;
  const Tile tile = tiles[blockIdx.x];
  const DevScene& sc = scenes[tile.scene];
  const int N = sc.n_obs;
  const int warps = blockDim.x >> 5;

  float* sW = smem;                                   // [3][NC][m]
  float4* sObs = reinterpret_cast<float4*>(smem + ((3 * NC * m + 3) & ~3));  // [N][2]
  float* sBuf = reinterpret_cast<float*>(sObs + 2 * N);                      // [warps][64]

  for (int i = threadIdx.x; i < 3 * NC * m; i += blockDim.x) sW[i] = c.basis32[i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double* o = obs + size_t(sc.obs_off + i) * 6;
    sObs[2 * i] = make_float4(float(o[0]), float(o[1]), float(o[2]), float(o[3]));
    sObs[2 * i + 1] = make_float4(float(1.0 / o[4]), float(1.0 / o[5]), float(o[4]), float(o[5]));
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= tile.count) return;
  const int j = layout[tile.scene].off + tile.first + warp;   // global sample index
  float* xbuf = sBuf + warp * 64;      // xi, slot layout
  float* vbuf = xbuf + 32;             // lambda + rho w, slot layout

  const float* W0 = sW;
  const float* W1 = sW + NC * m;
  const float* W2 = sW + 2 * NC * m;

  // ---- per-lane coefficient slot and its constant rows
  const int axis = lane >> 4, kk = lane & 15;
  const bool valid = kk < NC;
  float Mrow[NC], MProw[NC];
  float xibp = 0.f, lam = 0.f;
  const float b_ax0 = float(sc.ego[axis + 0]);   // position
  const float b_ax1 = float(sc.ego[axis + 2]);   // velocity
  const float b_ax2 = float(sc.ego[axis + 4]);   // acceleration
  {
    if (valid) {
      const float* row = c.pj32 + size_t((N * 2 + axis) * NC + kk) * (2 * NC + 3);
#pragma unroll
      for (int i = 0; i < NC; ++i) { Mrow[i] = row[i]; MProw[i] = row[NC + i]; }
      // Step 1: xi_bar = Gs p_axis + Hs b_axis (x uses the v_d entries, y the y_d entries)
      const float* s1 = c.s1_32 + size_t(axis * NC + kk) * (ns + 3);
      const double* pj = pin + size_t(j) * (2 * ns);
      float xb = 0.f;
      for (int q = 0; q < ns; ++q) xb += s1[q] * float(pj[(axis == 0 ? ns : 0) + q]);
      xb += s1[ns] * b_ax0 + s1[ns + 1] * b_ax1 + s1[ns + 2] * b_ax2;
      xbuf[lane] = xb;
      // constant part of the xi-step: M xi_bar + C b0 (needs all of xi_bar)
      xibp = row[2 * NC] * b_ax0 + row[2 * NC + 1] * b_ax1 + row[2 * NC + 2] * b_ax2;
    } else {
#pragma unroll
      for (int i = 0; i < NC; ++i) { Mrow[i] = 0.f; MProw[i] = 0.f; }
    }
    __syncwarp();
    if (valid) {
#pragma unroll
      for (int i = 0; i < NC; ++i) xibp += Mrow[i] * xbuf[axis * 16 + i];
    }
  }

  const float rho = float(prm.rho);
  const float hrho = 0.5f * rho;
  const float v_min = float(prm.v_min), v_max = float(prm.v_max), a_max = float(prm.a_max);
  const float kmax = float(prm.kappa_max), inv_kmax = float(1.0 / prm.kappa_max);
  const float c_max = float(prm.c_max);
  const float kr = float(fabs(sc.kappa_road));
  const float y_lb = float(sc.y_lb), y_ub = float(sc.y_ub);
  const float dt = float(prm.dt);

  float tt[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) tt[s] = float(s * 32 + lane) * dt;

  float da[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) da[s] = 0.f;

  float r_acc = 0.f, cu_acc = 0.f;

  for (int it = 0;; ++it) {
    __syncwarp();
    float xv[NC], yv[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) { xv[i] = xbuf[i]; yv[i] = xbuf[16 + i]; }

    // ---- A: kinematics at the lane's timesteps
    float px[SLOTS], py[SLOTS], vx[SLOTS], vy[SLOTS], ax[SLOTS], ay[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int t = s * 32 + lane;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
      if (t < m) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float w0 = W0[k * m + t], w1 = W1[k * m + t], w2 = W2[k * m + t];
          a0 = fmaf(w0, xv[k], a0); b0 = fmaf(w0, yv[k], b0);
          a1 = fmaf(w1, xv[k], a1); b1 = fmaf(w1, yv[k], b1);
          a2 = fmaf(w2, xv[k], a2); b2 = fmaf(w2, yv[k], b2);
        }
      }
      px[s] = a0; vx[s] = a1; ax[s] = a2; py[s] = b0; vy[s] = b1; ay[s] = b2;
    }

    if (it == prm.K) {
      // ---- scoring of xi^K (Alg. 1 line 9 and the Sec. V-A cost)
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int t = s * 32 + lane;
        if (t >= m) continue;
        float coll = 0.f;
        for (int i = 0; i < N; ++i) {
          const float4 o0 = sObs[2 * i], o1 = sObs[2 * i + 1];
          const float sx = (px[s] - fmaf(o0.z, tt[s], o0.x)) * o1.x;
          const float sy = (py[s] - fmaf(o0.w, tt[s], o0.y)) * o1.y;
          coll += fmaxf(0.f, 1.f - fmaf(sx, sx, sy * sy));
        }
        const float sp = sqrtf(fmaf(vx[s], vx[s], vy[s] * vy[s]));
        const float am = sqrtf(fmaf(ax[s], ax[s], ay[s] * ay[s]));
        const float kap = sp > 0.f ? (ay[s] * vx[s] - ax[s] * vy[s]) / (sp * sp * sp) : 0.f;
        r_acc += coll + fmaxf(0.f, sp - v_max) + fmaxf(0.f, am - a_max) +
                 fmaxf(0.f, fabsf(kap) - kmax) + fmaxf(0.f, vx[s] * vx[s] * kr - c_max) +
                 fmaxf(0.f, py[s] - y_ub) + fmaxf(0.f, y_lb - py[s]);
        const float dv = sp - v_max;
        cu_acc = fmaf(dv, dv, cu_acc);
      }
      break;
    }

    // ---- B: obstacle projection, accumulated residual sum_i (h_o,i - p)
    float ex[SLOTS], ey[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) { ex[s] = 0.f; ey[s] = 0.f; }
    for (int i = 0; i < N; ++i) {
      const float4 o0 = sObs[2 * i], o1 = sObs[2 * i + 1];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const float dx = px[s] - fmaf(o0.z, tt[s], o0.x);
        const float dy = py[s] - fmaf(o0.w, tt[s], o0.y);
        const float sx = dx * o1.x, sy = dy * o1.y;
        const float d2 = fmaf(sx, sx, sy * sy);
        if (d2 < 1.f) {
          if (d2 > 0.f) {
            const float g = rsqrtf(d2) - 1.f;
            ex[s] = fmaf(g, dx, ex[s]);
            ey[s] = fmaf(g, dy, ey[s]);
          } else {
            ex[s] += o1.z;      // atan2(0, 0) = 0: h = (x_o + a, y_o)
          }
        }
      }
    }

    // ---- C: velocity / acceleration / lane rows and the transposed contraction
    float wx[NC], wy[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) { wx[k] = 0.f; wy[k] = 0.f; }
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int t = s * 32 + lane;
      if (t >= m) continue;
      const float v2 = fmaf(vx[s], vx[s], vy[s] * vy[s]);
      float cv = 1.f, sv = 0.f, sp = 0.f;
      if (v2 > 0.f) { const float rv = rsqrtf(v2); cv = vx[s] * rv; sv = vy[s] * rv; sp = v2 * rv; }
      const float a2 = fmaf(ax[s], ax[s], ay[s] * ay[s]);
      float ca = 1.f, sa = 0.f, am = 0.f;
      if (a2 > 0.f) { const float ra = rsqrtf(a2); ca = ax[s] * ra; sa = ay[s] * ra; am = a2 * ra; }
      const float S = fabsf(sa * cv - ca * sv);               // |sin(alpha_a - alpha_v)|
      const float dap = (it == 0) ? fminf(am, a_max) : da[s];
      const float vmin_b = fmaxf(v_min, sqrtf(dap * S * inv_kmax));
      float vmax_b = v_max;
      if (kr > 0.f) {
        const float tc = kr * cv * cv;
        if (tc > 0.f) vmax_b = fminf(v_max, sqrtf(c_max / tc));
      }
      const float dv = fminf(fmaxf(sp, vmin_b), vmax_b);
      const float kd = dv * dv * kmax;
      const float amax_b = (S * a_max <= kd) ? a_max : kd / S;
      const float dan = fminf(am, amax_b);
      da[s] = dan;
      const float evx = fmaf(dv, cv, -vx[s]), evy = fmaf(dv, sv, -vy[s]);
      const float eax = fmaf(dan, ca, -ax[s]), eay = fmaf(dan, sa, -ay[s]);
      const float ely = fminf(fmaxf(py[s], y_lb), y_ub) - py[s];
      const float eoy = ey[s] + ely;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const float w0 = W0[k * m + t], w1 = W1[k * m + t], w2 = W2[k * m + t];
        wx[k] = fmaf(w0, ex[s], fmaf(w1, evx, fmaf(w2, eax, wx[k])));
        wy[k] = fmaf(w0, eoy, fmaf(w1, evy, fmaf(w2, eay, wy[k])));
      }
    }

    // ---- D: reduce, multipliers, xi-step
    const float wl = reduce_scatter<NC>(wx, wy, lane);
    if (valid) {
      if (it > 0) lam = fmaf(hrho, wl, lam);
      vbuf[lane] = fmaf(rho, wl, lam);
    }
    __syncwarp();
    if (valid) {
      float acc = xibp;
      const float* vb = vbuf + axis * 16;
#pragma unroll
      for (int i = 0; i < NC; ++i) acc = fmaf(Mrow[i], vb[i], acc);
#pragma unroll
      for (int i = 0; i < NC; ++i) acc = fmaf(MProw[i], axis ? yv[i] : xv[i], acc);
      xbuf[lane] = acc;
    }
  }

  // ---- outputs
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    r_acc += __shfl_xor_sync(kFull, r_acc, o);
    cu_acc += __shfl_xor_sync(kFull, cu_acc, o);
  }
  if (lane == 0) {
    r_out[j] = double(r_acc);
    cu_out[j] = double(cu_acc);
  }
  if (xi_out != nullptr && valid) xi_out[size_t(j) * 2 * NC + axis * NC + kk] = double(xbuf[lane]);
}

template <int NC, int SLOTS>
cudaError_t launch_t(const DevScene* scenes, const Layout* layout, const double* obs,
                     const Tile* tiles, int n_tiles, int warps, const double* p, const Consts& c,
                     const Params& prm, double* xi, double* r, double* cu, cudaStream_t s) {
  size_t shm = sizeof(float) * (((3 * NC * prm.m + 3) & ~3) + 8 * prm.max_obs + 64 * warps);
  fused_kernel<NC, SLOTS><<<n_tiles, warps * 32, shm, s>>>(scenes, layout, obs, tiles, p, c, prm,
                                                           xi, r, cu);
  return cudaGetLastError();
}

template <int NC, int SLOTS>
void set_attr() {
  cudaFuncSetAttribute(fused_kernel<NC, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       200 * 1024);
}

}  // namespace

void fused_setup() {
  set_attr<8, 4>(); set_attr<8, 8>();
  set_attr<11, 4>(); set_attr<11, 8>();
  set_attr<16, 4>(); set_attr<16, 8>();
}

bool fused_supported(int n, int m) {
  return (n == 8 || n == 11 || n == 16) && m >= 2 && m <= 256;
}

cudaError_t launch_fused_f32(const DevScene* scenes, const Layout* layout, const double* obs,
                             const Tile* tiles, int n_tiles, int warps, const double* p,
                             const Consts& c, const Params& prm, double* xi, double* r,
                             double* cu, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  const bool small = prm.m <= 128;
#define PLAN_FUSED_CASE(NC_)                                                                \
  if (prm.n == NC_)                                                                          \
    return small ? launch_t<NC_, 4>(scenes, layout, obs, tiles, n_tiles, warps, p, c, prm,  \
                                    xi, r, cu, s)                                            \
                 : launch_t<NC_, 8>(scenes, layout, obs, tiles, n_tiles, warps, p, c, prm,  \
                                    xi, r, cu, s);
  PLAN_FUSED_CASE(8)
  PLAN_FUSED_CASE(11)
  PLAN_FUSED_CASE(16)
#undef PLAN_FUSED_CASE
  return cudaErrorInvalidValue;
}

}  // namespace plan

// Tensor-core lower-level solve: Step 1, the K iterations of Alg. 2 and the
// scoring of Alg. 1 line 9, with the two n-wide contractions of every
// iteration on the 5th-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory) and the per-timestep projections on the CUDA cores.
//
// A CTA holds 8 samples of one scene; column c = 2 s + axis of the MMAs is
// (sample s, axis).  With delta = xi - xi_bar (the increment form of the
// fused FP32 kernel) one iteration is
//   forward    D_d[t][c] = sum_k W_d[t][k] delta[k][c]           d = 0, 1, 2
//              (Eq. param: position, velocity, acceleration rows; M = 128
//              timesteps, N = 16, K = n; lanes of tensor memory = timesteps)
//   projection per (t, c) on the CUDA cores: obstacles (Eqs. split_alpha_o,
//              clip_d_o), velocity and acceleration (Eqs. clip_d_v, clip_d_a),
//              lane slack (Eq. update_slack), giving the residual rows
//              R_d[t][c] of h - F xi and e - s - G xi,
//   transpose  g[k][c] = sum_d sum_t W_d[t][k] R_d[t][c]           (M = 64,
//              N = 16, K = 3 m; g = F^T (h - F xi) + G^T (e - s - G xi)),
//   update     lambda += rho/2 g (Eq. update_lagrange), and the xi-step of
//              Eq. split_xy in increment form delta += M (lambda + rho g - delta).
//
// Operand precision (plan_prec): TF32 (one pass, operands rounded to
// nearest), TF32X3 (operands split into a TF32 head and a TF32 tail,
// head*head + head*tail + tail*head: float32-level products), BF16 (one
// pass).  Accumulation is float32 in tensor memory in every mode.
//
// Operands sit in shared memory in the canonical no-swizzle K-major layout:
// 8-row x 16-byte core matrices, LBO = byte distance of core matrices along
// K, SBO = byte distance of 8-row groups.  The transposed contraction uses
// M = 64 with only rows 0..n-1 real: its A operand interleaves the two real
// row groups (SBO = 128, LBO = 256) so that row groups 2..7 read the next
// core matrices of the same buffer and produce rows that are ignored.  The
// residual operand uses LBO = 144 so that the per-timestep writes of 32
// lanes fall in 32 different banks.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace plan {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTcSamples = 8;             // samples per CTA
constexpr int kTcThreads = 256;           // 8 warps
constexpr int kTmemCols = 64;             // forward D: columns 0..47, transpose D: 48..63
constexpr uint32_t kColT = 48;
constexpr uint32_t kLboT = 256, kSboT = 128;   // transpose A operand (interleaved)
constexpr uint32_t kLboR = 144;                // residual operand
constexpr long long kWaitCycles = 2000000000ll;   // about one second at 2 GHz

template <int MODE>
struct Tc {
  static constexpr int EB = MODE == PLAN_PREC_BF16 ? 2 : 4;   // bytes per operand element
  static constexpr int EPC = 16 / EB;                         // elements per core-matrix row
  static constexpr int KI = 32 / EB;                          // K of one MMA instruction
  static constexpr int PASSES = MODE == PLAN_PREC_TF32X3 ? 3 : 1;
  static constexpr int COPIES = MODE == PLAN_PREC_TF32X3 ? 2 : 1;   // head (and tail)
  // instruction descriptor: D float32, A and B K-major, dense
  static constexpr uint32_t fmt = MODE == PLAN_PREC_BF16 ? 1u : 2u;
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(N >> 3) << 17) |
           (uint32_t(M >> 4) << 24);
  }
};

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Byte sizes of the operand buffers (one copy).
template <int NC, int MODE>
struct TcLayout {
  static constexpr int KP = round_up(NC, Tc<MODE>::KI);        // padded n
  static constexpr uint32_t SBO_F = uint32_t(KP / Tc<MODE>::EPC) * 128u;
  static constexpr uint32_t FWD_A = 16u * SBO_F;              // one derivative, 128 rows
  static constexpr uint32_t FWD_B = 2u * SBO_F;               // 16 columns
  __host__ __device__ static int mk(int m) { return round_up(m, Tc<MODE>::KI); }
  __host__ __device__ static int chunks(int m) { return 3 * mk(m) / Tc<MODE>::EPC; }
  __host__ __device__ static uint32_t tr_a(int m) { return uint32_t(chunks(m)) * kLboT + 1024u; }
  __host__ __device__ static uint32_t sbo_r(int m) { return uint32_t(chunks(m)) * kLboR; }
  __host__ __device__ static uint32_t tr_b(int m) { return 2u * sbo_r(m); }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (MODE == PLAN_PREC_BF16) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
  } else {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}

// Bounded wait for the phase `parity` of an mbarrier; false after `limit` SM
// clock cycles (about a second by default).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Diagnostic of the bounded wait: one thread waits for the first phase of an
// mbarrier that expects one arrival and gets none.  The wait gives up after
// `limit` cycles and the kernel raises the error flag the solve uses.
__global__ void wait_probe_kernel(long long limit, int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_addr(&bar), 0, limit)) atomicExch(err, 1);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
               "%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                 "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (row r, k) of a K-major operand.
template <int MODE>
__device__ __forceinline__ uint32_t op_off(int r, int k, uint32_t lbo, uint32_t sbo) {
  constexpr int EPC = Tc<MODE>::EPC, EB = Tc<MODE>::EB;
  return uint32_t(r >> 3) * sbo + uint32_t(k / EPC) * lbo + uint32_t(r & 7) * 16u +
         uint32_t(k % EPC) * EB;
}

// Store v at byte offset `off` of the head copy (and its tail at off + copy).
template <int MODE>
__device__ __forceinline__ void op_put(unsigned char* buf, uint32_t copy, uint32_t off, float v) {
  if constexpr (MODE == PLAN_PREC_BF16) {
    *reinterpret_cast<__nv_bfloat16*>(buf + off) = __float2bfloat16_rn(v);
  } else {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    *reinterpret_cast<uint32_t*>(buf + off) = h;
    if constexpr (MODE == PLAN_PREC_TF32X3)
      *reinterpret_cast<float*>(buf + copy + off) = v - __uint_as_float(h);
  }
}

__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

// Issue cost of the contractions of one Alg. 2 iteration at a wide N, for a
// CTA that would hold 64 samples (N = 128 columns = 64 samples x 2 axes) of
// the m = 200, n = 16 workload: TF32 MMAs (kind::tf32, `passes` 1 or 3 for
// the split mode), operands in shared memory, accumulators in tensor memory.
//   forward     3 derivatives x 2 row tiles (256 timesteps) x 2 K steps (n =
//               16), M = 128, N = 128: D[t][c] in columns 0..383, one commit
//               and wait per row tile;
//   transposed  K = 3 x 256 = 768 (96 K steps) either as M = 128 (columns) x
//               N = 16 (coefficients), or as M = 64 (16 coefficients padded) x
//               N = 128 (columns); each with one accumulator, and again with
//               the K steps dealt round-robin to four accumulators (partial
//               sums a kernel would add afterwards), so that consecutive MMAs
//               do not depend on one another.
// Only the MMAs are timed: the operand values are zeros and the results are
// not read; the K-step operands cycle through 8 staged chunks.  Thread 0
// issues and waits (bounded); out[kProbeParts * cta + q] = SM cycles per
// iteration of part q.  The paper has no counterpart: this measures whether B x (basis) is
// dense enough for the tensor cores on this part.
constexpr int kProbeThreads = 128;
constexpr int kProbeParts = 5;
constexpr uint32_t kProbeCols = 512;

__global__ void __launch_bounds__(kProbeThreads, 1)
tc_wide_probe_kernel(int passes, int iters, double* out, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  // canonical no-swizzle K-major operands: [8-row group][16-byte K chunk][8 rows][16 B]
  unsigned char* aF = dsm;                // 128 rows x K 16:  8 KB (SBO 512)
  unsigned char* bF = aF + 8192;          // 128 rows x K 16:  8 KB
  unsigned char* aT1 = bF + 8192;         // 128 rows x K 64: 32 KB (SBO 2048)
  unsigned char* bT1 = aT1 + 32768;       //  16 rows x K 64:  4 KB
  unsigned char* aT2 = bT1 + 4096;        //  64 rows x K 64: 16 KB
  unsigned char* bT2 = aT2 + 16384;       // 128 rows x K 64: 32 KB
  const uint32_t bytes = 8192u + 8192u + 32768u + 4096u + 16384u + 32768u;
  for (uint32_t i = tid; i < bytes / 16; i += kProbeThreads)
    reinterpret_cast<uint4*>(dsm)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tslot)), "r"(kProbeCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    using T = Tc<PLAN_PREC_TF32>;
    const uint32_t bar = smem_addr(&mbar);
    const uint32_t idF = T::idesc(128, 128), id1 = T::idesc(128, 16), id2 = T::idesc(64, 128);
    const uint32_t sF = smem_addr(aF), sFB = smem_addr(bF);
    const uint32_t s1 = smem_addr(aT1), s1B = smem_addr(bT1);
    const uint32_t s2 = smem_addr(aT2), s2B = smem_addr(bT2);
    uint32_t phase = 0;
    long long c_f = 0, c_1 = 0, c_2 = 0, c_3 = 0, c_4 = 0;
    bool ok = true;
    for (int it = 0; it < iters && ok; ++it) {
      const long long t0 = clock64();
      for (int tile = 0; tile < 2 && ok; ++tile) {
        fence_after();
        for (int d = 0; d < 3; ++d)
          for (int ks = 0; ks < 2; ++ks)
            for (int ps = 0; ps < passes; ++ps)
              mma<PLAN_PREC_TF32>(tmem + 128u * d, sdesc(sF + ks * 256u, 128u, 512u),
                                  sdesc(sFB + ks * 256u, 128u, 512u), idF, (ks | ps) != 0);
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
      }
      const long long t1 = clock64();
      if (ok) {
        fence_after();
        for (int ks = 0; ks < 96; ++ks)
          for (int ps = 0; ps < passes; ++ps)
            mma<PLAN_PREC_TF32>(tmem + 384u, sdesc(s1 + (ks & 7) * 256u, 128u, 2048u),
                                sdesc(s1B + (ks & 7) * 256u, 128u, 2048u), id1, (ks | ps) != 0);
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
      }
      const long long t2 = clock64();
      if (ok) {
        fence_after();
        for (int ks = 0; ks < 96; ++ks)
          for (int ps = 0; ps < passes; ++ps)
            mma<PLAN_PREC_TF32>(tmem + 384u, sdesc(s2 + (ks & 7) * 256u, 128u, 2048u),
                                sdesc(s2B + (ks & 7) * 256u, 128u, 2048u), id2, (ks | ps) != 0);
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
      }
      const long long t3 = clock64();
      if (ok) {    // four accumulators of N = 16 (columns 384 .. 447)
        fence_after();
        for (int ks = 0; ks < 96; ++ks)
          for (int ps = 0; ps < passes; ++ps)
            mma<PLAN_PREC_TF32>(tmem + 384u + 16u * (ks & 3), sdesc(s1 + (ks & 7) * 256u, 128u, 2048u),
                                sdesc(s1B + (ks & 7) * 256u, 128u, 2048u), id1, (ks >= 4) | (ps != 0));
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
      }
      const long long t4 = clock64();
      if (ok) {    // four accumulators of N = 128 (all 512 columns)
        fence_after();
        for (int ks = 0; ks < 96; ++ks)
          for (int ps = 0; ps < passes; ++ps)
            mma<PLAN_PREC_TF32>(tmem + 128u * (ks & 3), sdesc(s2 + (ks & 7) * 256u, 128u, 2048u),
                                sdesc(s2B + (ks & 7) * 256u, 128u, 2048u), id2, (ks >= 4) | (ps != 0));
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
        phase ^= 1u;
      }
      const long long t5 = clock64();
      c_f += t1 - t0;
      c_1 += t2 - t1;
      c_2 += t3 - t2;
      c_3 += t4 - t3;
      c_4 += t5 - t4;
    }
    if (!ok) atomicExch(err, 1);
    double* o = out + kProbeParts * blockIdx.x;
    o[0] = double(c_f) / iters;
    o[1] = double(c_1) / iters;
    o[2] = double(c_2) / iters;
    o[3] = double(c_3) / iters;
    o[4] = double(c_4) / iters;
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kProbeCols));
  }
}

template <int NC, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_kernel(const DevScene* __restrict__ scenes, const Layout* __restrict__ layout,
          const double* __restrict__ obs, const Tile* __restrict__ tiles,
          const double* __restrict__ pin, Consts c, Params prm, double* __restrict__ xi_out,
          double* __restrict__ r_out, double* __restrict__ cu_out, int* __restrict__ st_out,
          int* __restrict__ err) {
  using T = Tc<MODE>;
  using LY = TcLayout<NC, MODE>;
  constexpr int NCP = basis32_ncp(NC);
  constexpr int ST = basis32_stride(NC);
  constexpr int KP = LY::KP;
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ float sXb[16][17];           // xi_bar[c][k]
  __shared__ float sG[16][17];            // g[c][k] of the transpose
  __shared__ float sM[2][kMaxCoef][kMaxCoef + 1];     // rows padded: conflict-free row reads
  __shared__ float sMoved[kTcSamples];
  __shared__ float sScore[8][4][2];
  __shared__ float sIab[2];
  __shared__ int sBadXi[kTcSamples];      // a coefficient of the sample's solution is not finite

  const int m = prm.m, ns = prm.n_seg;
  const int mK = LY::mk(m);
  const Tile tile = tiles[blockIdx.x];
  const DevScene& sc = scenes[tile.scene];
  const int N = sc.n_obs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- shared memory carve-up
  const uint32_t cpF = 3u * LY::FWD_A, cpFB = LY::FWD_B;
  const uint32_t cpT = LY::tr_a(m), cpR = LY::tr_b(m), sboR = LY::sbo_r(m);
  unsigned char* bFA = dsm;                                   // forward A, COPIES x 3 derivatives
  unsigned char* bTA = bFA + T::COPIES * cpF;                 // transpose A
  unsigned char* bFB = bTA + T::COPIES * cpT;                 // forward B (delta)
  unsigned char* bTB = bFB + T::COPIES * cpFB;                // transpose B (residual rows)
  float4* sObs = reinterpret_cast<float4*>(bTB + T::COPIES * cpR);   // [N][4]
  float* sThr = reinterpret_cast<float*>(sObs + 4 * N);      // [8 warps][4 samples][N]
  const uint32_t opBytes = uint32_t(reinterpret_cast<unsigned char*>(sObs) - dsm);

  for (uint32_t i = tid; i < opBytes / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(dsm)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // W_d[t][k] as the forward A (rows t) and the transpose A (rows k, K = d mK + t)
  for (int e = tid; e < 3 * 128 * KP; e += kTcThreads) {
    const int d = e / (128 * KP), t = (e / KP) % 128, k = e % KP;
    const float w = (t < m && k < NC) ? c.basis32[size_t(t) * ST + d * NCP + k] : 0.f;
    op_put<MODE>(bFA + d * LY::FWD_A, cpF, op_off<MODE>(t, k, 128u, LY::SBO_F), w);
    if (k < 16 && t < mK) op_put<MODE>(bTA, cpT, op_off<MODE>(k, d * mK + t, kLboT, kSboT), w);
  }
  for (int i = tid; i < N; i += kTcThreads) {
    const double* o = obs + size_t(sc.obs_off + i) * 6;
    const double ia = 1.0 / o[4], ib = 1.0 / o[5];
    const float nx0 = float(-o[0] * ia), nvx = float(-o[2] * ia * prm.dt);
    const float ny0 = float(-o[1] * ib), nvy = float(-o[3] * ib * prm.dt);
    sObs[4 * i + 0] = make_float4(nx0, nx0, nvx, nvx);
    sObs[4 * i + 1] = make_float4(ny0, ny0, nvy, nvy);
    sObs[4 * i + 2] = make_float4(float(ia), float(ia), float(ib), float(ib));
    sObs[4 * i + 3] = make_float4(float(o[4]), float(o[5]), 0.f, 0.f);
  }
  for (int e = tid; e < 8 * 4 * N; e += kTcThreads) sThr[e] = -3.0e38f;
  for (int e = tid; e < 2 * kMaxCoef * kMaxCoef; e += kTcThreads) {
    const int ax_ = e / (kMaxCoef * kMaxCoef), k_ = (e / kMaxCoef) % kMaxCoef, i_ = e % kMaxCoef;
    sM[ax_][k_][i_] = (k_ < NC && i_ < NC)
                          ? c.pj32[size_t((N * 2 + ax_) * NC + k_) * (2 * NC + c.ne) + i_]
                          : 0.f;
  }
  if (tid < kTcSamples) { sMoved[tid] = 0.f; sBadXi[tid] = 0; }
  if (warp == 0) {
    float ia_max = 0.f, ib_max = 0.f;
    for (int i = lane; i < N; i += 32) {
      const double* o = obs + size_t(sc.obs_off + i) * 6;
      ia_max = fmaxf(ia_max, float(1.0 / o[4]));
      ib_max = fmaxf(ib_max, float(1.0 / o[5]));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      ia_max = fmaxf(ia_max, __shfl_xor_sync(kFull, ia_max, o));
      ib_max = fmaxf(ib_max, __shfl_xor_sync(kFull, ib_max, o));
    }
    if (lane == 0) { sIab[0] = ia_max; sIab[1] = ib_max; }
  }

  // ---- (column, coefficient) slot of this thread for Step 1 and the update
  const int col = tid >> 4, kk = tid & 15;
  const int cs = col >> 1, caxis = col & 1;
  const bool slot = kk < NC && cs < tile.count;
  const int jcol = layout[tile.scene].off + tile.first + cs;   // sample of this column
  float xb_l = 0.f;
  if (slot) {
    // xi_bar = Gs p_axis + Hs b_axis in float64 (Step 1, Eq. over_3); with goal
    // entries b_axis also holds x_f (x) or y_f (y)
    const double* s1 = c.s1_64 + size_t(caxis * NC + kk) * (ns + c.ne);
    const double* pj = pin + size_t(jcol) * prm.d_p;
    double xb = 0.0;
    for (int q = 0; q < ns; ++q) xb = fma(s1[q], pj[(caxis == 0 ? ns : 0) + q], xb);
    xb = fma(s1[ns], sc.ego[caxis], xb);
    xb = fma(s1[ns + 1], sc.ego[caxis + 2], xb);
    xb = fma(s1[ns + 2], sc.ego[caxis + 4], xb);
    if (prm.goal) xb = fma(s1[ns + 3], pj[2 * ns + caxis], xb);
    xb_l = float(xb);
  }
  sXb[col][kk] = xb_l;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tslot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  const uint32_t bar = smem_addr(&mbar);

  // ---- timestep slot of this thread for the projections
  const int quarter = warp & 3, sgrp = warp >> 2;
  const int t = 32 * quarter + lane;
  const int tcl = min(t, m - 1);
  const float tt = float(t);
  const float act = t < m ? 1.f : 0.f;
  float A[4];
#pragma unroll
  for (int sl = 0; sl < 4; ++sl) A[sl] = (4 * sgrp + sl < tile.count) ? act : 0.f;

  // reference kinematics at xi_bar: ref[sl][2 d + axis]
  float ref[4][6];
  {
    const float* row = c.basis32 + size_t(tcl) * ST;
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      const int cx = 8 * sgrp + 2 * sl;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const float w = row[d * NCP + k];
          ax_ = fmaf(w, sXb[cx][k], ax_);
          ay_ = fmaf(w, sXb[cx + 1][k], ay_);
        }
        ref[sl][2 * d] = ax_;
        ref[sl][2 * d + 1] = ay_;
      }
    }
  }

  const float rho = float(prm.rho), hrho = 0.5f * rho;
  const float v_min = float(prm.v_min), v_max = float(prm.v_max), a_max = float(prm.a_max);
  const float kmax = float(prm.kappa_max), inv_kmax = float(1.0 / prm.kappa_max);
  const float c_max = float(prm.c_max);
  const float kr = float(fabs(sc.kappa_road));
  const float y_lb = float(sc.y_lb), y_ub = float(sc.y_ub);
  const float iab = sIab[caxis];
  const float* Mrow = &sM[caxis][kk][0];

  float da[4] = {0.f, 0.f, 0.f, 0.f};
  // road profile: curvature at the previous iterate (Eq. clip_d_v), lane limits
  // at the current one; without a profile both are the scene's constants
  const bool road = sc.n_road > 0;
  float xprev[4] = {0.f, 0.f, 0.f, 0.f};
  float lam = 0.f, dl = 0.f;
  float r_acc[4] = {0.f, 0.f, 0.f, 0.f}, cu_acc[4] = {0.f, 0.f, 0.f, 0.f};
  float* thr = sThr + warp * 4 * N;
  uint32_t phase = 0;
  bool failed = false;
  const uint32_t idF = T::idesc(128, 16), idT = T::idesc(64, 16);
  const uint32_t aF = smem_addr(bFA), aT = smem_addr(bTA), aFB = smem_addr(bFB), aTB = smem_addr(bTB);
  const int ksF = KP / T::KI, ksT = 3 * mK / T::KI;

  for (int it = 0;; ++it) {
    // ---- forward contraction (delta = 0 at it = 0)
    float kd[3][8];
    if (it > 0) {
      bool ok = true;
      if (tid == 0) {
        fence_after();
#pragma unroll
        for (int d = 0; d < 3; ++d)
          for (int ks = 0; ks < ksF; ++ks)
#pragma unroll
            for (int ps = 0; ps < T::PASSES; ++ps) {
              const uint32_t a = aF + (ps == 2 ? cpF : 0u) + d * LY::FWD_A + ks * 256u;
              const uint32_t b = aFB + (ps == 1 ? cpFB : 0u) + ks * 256u;
              mma<MODE>(tmem + 16u * d, sdesc(a, 128u, LY::SBO_F), sdesc(b, 128u, LY::SBO_F), idF,
                        (ks | ps) != 0);
            }
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
      }
      phase ^= 1u;
      if (__syncthreads_or(!ok)) { failed = true; break; }
      fence_after();
      const uint32_t ta = tmem + (uint32_t(32 * quarter) << 16) + 8u * sgrp;
      tmem_ld8(ta, kd[0]);
      tmem_ld8(ta + 16u, kd[1]);
      tmem_ld8(ta + 32u, kd[2]);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int i = 0; i < 8; ++i) kd[d][i] = 0.f;
    }

    float px[4], py[4], vx[4], vy[4], ax[4], ay[4];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      px[sl] = ref[sl][0] + kd[0][2 * sl]; py[sl] = ref[sl][1] + kd[0][2 * sl + 1];
      vx[sl] = ref[sl][2] + kd[1][2 * sl]; vy[sl] = ref[sl][3] + kd[1][2 * sl + 1];
      ax[sl] = ref[sl][4] + kd[2][2 * sl]; ay[sl] = ref[sl][5] + kd[2][2 * sl + 1];
    }

    if (it == prm.K) {
      // ---- scoring of xi^K (Alg. 1 line 9 and the Sec. V-A cost)
#pragma unroll
      for (int sl = 0; sl < 4; ++sl) {
        float coll = 0.f;
        for (int i = 0; i < N; ++i) {
          const float4 q0 = sObs[4 * i], q1 = sObs[4 * i + 1], q2 = sObs[4 * i + 2];
          const float sx = fmaf(px[sl], q2.x, fmaf(q0.z, tt, q0.x));
          const float sy = fmaf(py[sl], q2.z, fmaf(q1.z, tt, q1.x));
          coll += fmaxf(0.f, 1.f - fmaf(sx, sx, sy * sy));
        }
        const float sp = fast_sqrt(fmaf(vx[sl], vx[sl], vy[sl] * vy[sl]));
        const float am = fast_sqrt(fmaf(ax[sl], ax[sl], ay[sl] * ay[sl]));
        const float kap =
            sp > 0.f ? __fdividef(ay[sl] * vx[sl] - ax[sl] * vy[sl], sp * sp * sp) : 0.f;
        float kro = kr, ylo = y_lb, yup = y_ub;
        if (road) {
          road_eval<float>(sc, px[sl], &kro, &ylo, &yup);
          kro = fabsf(kro);
        }
        const float rt = coll + fmaxf(0.f, sp - v_max) + fmaxf(0.f, am - a_max) +
                         fmaxf(0.f, fabsf(kap) - kmax) + fmaxf(0.f, vx[sl] * vx[sl] * kro - c_max) +
                         fmaxf(0.f, py[sl] - yup) + fmaxf(0.f, ylo - py[sl]);
        const float dv = sp - v_max;
        r_acc[sl] = A[sl] * rt;
        cu_acc[sl] = A[sl] * dv * dv;
      }
      break;
    }

    // ---- projections and residual rows, one sample at a time
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
      const int s = 4 * sgrp + sl;
      const float mv = sMoved[s];
      float* th = thr + sl * N;
      float ex = 0.f, ey = 0.f;
      for (int i0 = 0; i0 < N; i0 += 32) {
        const int nc = min(32, N - i0);
        unsigned ins = 0u;
        // obstacles that may be within reach of this warp's points (exact skip)
        unsigned near = __ballot_sync(kFull, lane < nc && th[i0 + lane] - mv <= 1.001f);
        while (near) {
          const int ii = __ffs(near) - 1;
          near &= near - 1u;
          const float4 q0 = sObs[4 * (i0 + ii)], q1 = sObs[4 * (i0 + ii) + 1];
          const float4 q2 = sObs[4 * (i0 + ii) + 2];
          const float sx = fmaf(px[sl], q2.x, fmaf(q0.z, tt, q0.x));
          const float sy = fmaf(py[sl], q2.z, fmaf(q1.z, tt, q1.x));
          const float d2 = fmaf(sx, sx, sy * sy);
          ins |= (d2 < 1.f ? 1u : 0u) << ii;
          float dmin = A[sl] > 0.f ? d2 : 3.0e38f;
          dmin = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(dmin)));
          if (lane == 0) th[i0 + ii] = fast_sqrt(dmin) + mv;
        }
        ins = A[sl] > 0.f ? ins : 0u;
        unsigned uni = __reduce_or_sync(kFull, ins);
        while (uni) {
          const int ii = __ffs(uni) - 1;
          uni &= uni - 1u;
          if ((ins >> ii) & 1u) {
            const float4 q0 = sObs[4 * (i0 + ii)], q1 = sObs[4 * (i0 + ii) + 1];
            const float4 q2 = sObs[4 * (i0 + ii) + 2], q3 = sObs[4 * (i0 + ii) + 3];
            const float sx = fmaf(px[sl], q2.x, fmaf(q0.z, tt, q0.x));
            const float sy = fmaf(py[sl], q2.z, fmaf(q1.z, tt, q1.x));
            const float d2 = fmaf(sx, sx, sy * sy);
            if (d2 > 0.f) {
              const float gcorr = rsqrtf(d2) - 1.f;
              ex = fmaf(gcorr * q3.x, sx, ex);
              ey = fmaf(gcorr * q3.y, sy, ey);
            } else {
              ex += q3.x;     // atan2(0, 0) = 0: h = (x_o + a, y_o)
            }
          }
        }
      }

      const float v2 = fmaf(vx[sl], vx[sl], vy[sl] * vy[sl]);
      const bool vp = v2 > 0.f;
      const float rv = rsqrtf(v2);
      const float cv = vp ? vx[sl] * rv : 1.f, sv = vp ? vy[sl] * rv : 0.f, sp = vp ? v2 * rv : 0.f;
      const float a2 = fmaf(ax[sl], ax[sl], ay[sl] * ay[sl]);
      const bool ap = a2 > 0.f;
      const float ra = rsqrtf(a2);
      const float ca = ap ? ax[sl] * ra : 1.f, sa = ap ? ay[sl] * ra : 0.f, am = ap ? a2 * ra : 0.f;
      const float S = fabsf(sa * cv - ca * sv);               // |sin(alpha_a - alpha_v)|
      const float dap = (it == 0) ? fminf(am, a_max) : da[sl];
      const float vmin_b = fmaxf(v_min, fast_sqrt(dap * S * inv_kmax));
      float vmax_b = v_max;
      float krs = kr, ylbs = y_lb, yubs = y_ub;
      if (road) {
        float unused;
        road_eval<float>(sc, it == 0 ? px[sl] : xprev[sl], &krs, &unused, &unused);
        krs = fabsf(krs);
        road_eval<float>(sc, px[sl], &unused, &ylbs, &yubs);
        xprev[sl] = px[sl];
      }
      if (krs > 0.f) {
        const float tc = krs * cv * cv;
        if (tc > 0.f) vmax_b = fminf(v_max, fast_sqrt(__fdividef(c_max, tc)));
      }
      const float dv = fminf(fmaxf(sp, vmin_b), vmax_b);
      const float kdv = dv * dv * kmax;
      const float amax_b = (S * a_max <= kdv) ? a_max : __fdividef(kdv, S);
      const float dan = fminf(am, amax_b);
      da[sl] = dan;
      const float a_ = A[sl];
      const float rows[6] = {a_ * ex,
                             a_ * (ey + fminf(fmaxf(py[sl], ylbs), yubs) - py[sl]),
                             a_ * fmaf(dv, cv, -vx[sl]), a_ * fmaf(dv, sv, -vy[sl]),
                             a_ * fmaf(dan, ca, -ax[sl]), a_ * fmaf(dan, sa, -ay[sl])};
      if (t < mK) {
        const int cx = 8 * sgrp + 2 * sl;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          op_put<MODE>(bTB, cpR, op_off<MODE>(cx, d * mK + t, kLboR, sboR), rows[2 * d]);
          op_put<MODE>(bTB, cpR, op_off<MODE>(cx + 1, d * mK + t, kLboR, sboR), rows[2 * d + 1]);
        }
      }
    }

    // ---- transposed contraction g = sum_d W_d^T R_d
    fence_async_smem();
    fence_before();
    __syncthreads();
    {
      bool ok = true;
      if (tid == 0) {
        fence_after();
        for (int ks = 0; ks < ksT; ++ks)
#pragma unroll
          for (int ps = 0; ps < T::PASSES; ++ps) {
            const uint32_t a = aT + (ps == 2 ? cpT : 0u) + ks * (2u * kLboT);
            const uint32_t b = aTB + (ps == 1 ? cpR : 0u) + ks * (2u * kLboR);
            mma<MODE>(tmem + kColT, sdesc(a, kLboT, kSboT), sdesc(b, kLboR, sboR), idT,
                      (ks | ps) != 0);
          }
        mma_commit(bar);
        ok = mbar_wait(bar, phase);
      }
      phase ^= 1u;
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
    fence_after();
    if (warp == 0) {
      float gv[16];
      tmem_ld16(tmem + kColT, gv);     // lanes 0..15 hold rows k = 0..15
      tmem_wait_ld();
      if (lane < NC) {
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) sG[cc][lane] = gv[cc];
      }
    }
    fence_before();
    __syncthreads();

    // ---- multipliers and xi-step in increment form, slot (col, kk)
    float u = 0.f;
    if (slot) {
      const float wl = sG[col][kk];
      if (it > 0) lam = fmaf(hrho, wl, lam);
      u = fmaf(rho, wl, lam) - dl;
    }
    float step = 0.f;
#pragma unroll
    for (int k2 = 0; k2 < NC; ++k2)
      step = fmaf(Mrow[k2], __shfl_sync(kFull, u, (lane & 16) | k2), step);
    if (slot) {
      dl += step;
      op_put<MODE>(bFB, cpFB, op_off<MODE>(col, kk, 128u, LY::SBO_F), dl);
    }
    {
      // scaled bound on how far any point of sample cs moves in this step
      const float mvb = slot ? fabsf(step) * iab : 0.f;
      const float mx = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(mvb)));
      if (lane == 0) sMoved[cs] += 1.41422f * mx;
    }
    fence_async_smem();
    __syncthreads();
  }

  // ---- outputs
  if (!failed) {
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        r_acc[sl] += __shfl_xor_sync(kFull, r_acc[sl], o);
        cu_acc[sl] += __shfl_xor_sync(kFull, cu_acc[sl], o);
      }
      if (lane == 0) { sScore[warp][sl][0] = r_acc[sl]; sScore[warp][sl][1] = cu_acc[sl]; }
    }
  }
  if (slot && !(isfinite(xb_l) && isfinite(dl))) sBadXi[cs] = 1;
  __syncthreads();
  if (tid < kTcSamples && tid < tile.count) {
    const int g4 = tid >> 2, sl = tid & 3;
    const int j = layout[tile.scene].off + tile.first + tid;
    float rs = 0.f, cs_ = 0.f;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) { rs += sScore[4 * g4 + qq][sl][0]; cs_ += sScore[4 * g4 + qq][sl][1]; }
    r_out[j] = failed ? __longlong_as_double(0x7ff8000000000000ll) : double(rs);
    cu_out[j] = failed ? __longlong_as_double(0x7ff8000000000000ll) : double(cs_);
    if (st_out != nullptr)
      st_out[j] = (failed || sBadXi[tid] || !isfinite(rs) || !isfinite(cs_)) ? PLAN_ENONFINITE
                                                                               : PLAN_OK;
  }
  if (xi_out != nullptr && slot)
    xi_out[size_t(jcol) * 2 * NC + caxis * NC + kk] = double(xb_l) + double(dl);
  if (failed && tid == 0) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
  }
}

template <int NC, int MODE>
size_t tc_smem(const Params& prm) {
  using LY = TcLayout<NC, MODE>;
  constexpr int CP = Tc<MODE>::COPIES;
  return size_t(CP) * (3u * LY::FWD_A + LY::tr_a(prm.m) + LY::FWD_B + LY::tr_b(prm.m)) +
         size_t(64) * prm.max_obs + size_t(8 * 4 * 4) * prm.max_obs;
}

template <int NC, int MODE>
cudaError_t tc_launch(const DevScene* scenes, const Layout* layout, const double* obs,
                      const Tile* tiles, int n_tiles, const double* p, const Consts& c,
                      const Params& prm, double* xi, double* r, double* cu, int* st, int* err,
                      cudaStream_t s) {
  const size_t bytes = tc_smem<NC, MODE>(prm);
  tc_kernel<NC, MODE><<<n_tiles, kTcThreads, bytes, s>>>(scenes, layout, obs, tiles, p, c, prm, xi,
                                                          r, cu, st, err);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t tc_launch_mode(const DevScene* scenes, const Layout* layout, const double* obs,
                           const Tile* tiles, int n_tiles, const double* p, const Consts& c,
                           const Params& prm, double* xi, double* r, double* cu, int* st, int* err,
                           cudaStream_t s) {
  if (prm.n == 8) return tc_launch<8, MODE>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  if (prm.n == 11) return tc_launch<11, MODE>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  if (prm.n == 16) return tc_launch<16, MODE>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  return cudaErrorInvalidValue;
}

template <int MODE>
void tc_attr_mode() {
  constexpr int kMaxDyn = 200 * 1024;
  cudaFuncSetAttribute(tc_kernel<8, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
  cudaFuncSetAttribute(tc_kernel<11, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
  cudaFuncSetAttribute(tc_kernel<16, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
}

}  // namespace

void tc_setup() {
  tc_attr_mode<PLAN_PREC_TF32>();
  tc_attr_mode<PLAN_PREC_BF16>();
  tc_attr_mode<PLAN_PREC_TF32X3>();
}

bool tc_supported(int n, int m, int max_obs) {
  if (!(n == 8 || n == 11 || n == 16) || m < 2 || m > 128 || max_obs > kMaxObs) return false;
  Params prm{};
  prm.m = m;
  prm.max_obs = max_obs;
  return tc_smem<16, PLAN_PREC_TF32X3>(prm) <= size_t(200 * 1024);
}

int tc_samples_per_cta() { return kTcSamples; }

cudaError_t wait_probe(long long limit, cudaStream_t s, int* timed_out) {
  *timed_out = 0;
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return e;
  int h = 0;
  e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_probe_kernel<<<1, 32, 0, s>>>(limit, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  *timed_out = h;
  return e;
}

cudaError_t tc_wide_probe(int passes, int iters, int ctas, double* cycles, cudaStream_t s,
                          int* timed_out) {
  *timed_out = 0;
  double* d = nullptr;
  int* flag = nullptr;
  // 120 KB of dynamic shared memory keeps one probe CTA per SM
  constexpr size_t kProbeSmem = 120 * 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_wide_probe_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(kProbeSmem));
  if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(double) * kProbeParts * ctas);
  if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    tc_wide_probe_kernel<<<ctas, kProbeThreads, kProbeSmem, s>>>(passes, iters, d, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cycles, d, sizeof(double) * kProbeParts * ctas, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(timed_out, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  cudaFree(flag);
  return e;
}

cudaError_t launch_tc(int prec, const DevScene* scenes, const Layout* layout, const double* obs,
                      const Tile* tiles, int n_tiles, const double* p, const Consts& c,
                      const Params& prm, double* xi, double* r, double* cu, int* st, int* err,
                      cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  if (prec == PLAN_PREC_TF32)
    return tc_launch_mode<PLAN_PREC_TF32>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  if (prec == PLAN_PREC_TF32X3)
    return tc_launch_mode<PLAN_PREC_TF32X3>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  if (prec == PLAN_PREC_BF16)
    return tc_launch_mode<PLAN_PREC_BF16>(scenes, layout, obs, tiles, n_tiles, p, c, prm, xi, r, cu, st, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace plan

// Device kernels of libdpinn (sm_103a).
//
// One persistent, grouped kernel (`k_pinn`) processes a work list of
// (net, point-chunk) items for every subdomain net of the decomposition in a
// single launch.  Per chunk it runs, for tiles of P points:
//
//   forward  - jets (value, d/dx_q for every input, spatial Laplacian) through
//              the tanh MLP (Sec. 2.1, Eq. (2)); hidden-layer products are
//              dense (P*C) x W x W FP32 contractions, register-tiled, with the
//              tanh-jet recursion fused into the epilogue;
//   loss     - Navier-Stokes residuals (Eqs. (7)-(10)) and L_PDE (Eq. (5)),
//              or L_obs (Eq. (3)), or the ghost terms (Eqs. (13)-(14)) with
//              the anchor-normalised neighbour pressure (Eq. (15)) and the
//              asymmetric weights of Eq. (16);
//   reverse  - hand-written adjoint through residual, jets and layers;
//              weight gradients accumulate per work item (deterministic).
//
// The same kernel, without the reverse pass, evaluates the neighbour
// messages of Algorithm 1 (face values and master anchor values) and serves
// queries (values, or values + residuals, with the anchored pressure of
// Eq. (18)).
//
// Shared memory holds two activation buffers [W][RS] (RS = P*C padded so that
// rows fall on distinct banks), one weight matrix staged by a TMA bulk copy
// (cp.async.bulk + mbarrier), and small per-net tensors.  For every layer the
// jets (tanh value, first derivatives and Laplacian of the pre-activation)
// are stashed per thread (coalesced) in a per-CTA global scratch and re-read
// in the reverse pass, which therefore evaluates no tanh.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dk {

constexpr int NT = 256;     // threads per CTA of the grouped kernel
constexpr int MAXL = 16;    // maximum hidden layers

enum { K_PDE = 0, K_OBS = 1, K_FACE = 2, K_EVAL = 3, K_EVAL_ANC = 4, K_QUERY = 5 };
enum { M_TRAIN = 0, M_EVAL = 1, M_QUERY = 2 };
enum { ERR_TIMEOUT = 0, ERR_NONFINITE = 1, ERR_DOMAIN = 2 };

struct Shape {
  int ds, unst, din, dout, W, L;
  int npp;                     // padded per-net parameter stride (floats)
  int nTp;                     // per-net stride of the transposed hidden weights
  int twp;                     // 0: thetaT holds W_l^T (W x W); > 0: the streamed-weight layout of
                               // padded width twp (wide_pos below), a forward block W_l^T and a
                               // reverse block W_l per hidden layer, each W rows of twp floats
  int woff[MAXL + 1], boff[MAXL + 1];
  int act;                     // ACT_TANH or ACT_SIN
  float nu, p_ref;
  float anchor[3];
  float lam_obs, lam_pde, lam_gh_u, lam_time;
  float comp_w[3];
  float lam_gh_r, lam_gh_c1;   // interface residual and C1 matching (0 = off)
};

// loss numerators per work item: obs, PDE, gh_u, gh_p space, gh_p time,
// gh_r (residual matching), gh_c1 (first-derivative matching)
constexpr int LP = 7;

// Column position of neuron n in a row of the streamed-weight layout of
// padded width WP (a multiple of 32).  Lane l of a warp owns the neurons
// l + 32 m, m < WP / 32; the row holds them lane-blocked so that a lane reads
// its neurons' entries with vector loads: m = 4a + r (a < WP / 128) at
// 128 a + 4 l + r (float4 groups), the next two m (if there are two left) at
// a float2 block of 64, the last odd m at a block of 32.  A bijection of
// [0, WP).
__host__ __device__ constexpr int wide_pos(int n, int WP) {
  const int m = n >> 5, l = n & 31, tmg = WP / 32, g4 = tmg / 4, rem = tmg - 4 * g4;
  if (m < 4 * g4) return (m >> 2) * 128 + l * 4 + (m & 3);
  if (rem >= 2 && m < 4 * g4 + 2) return g4 * 128 + l * 2 + (m - 4 * g4);
  return g4 * 128 + (rem >= 2 ? 64 : 0) + l;
}

struct NetInfo {
  float center[4], scale[4];
  float inv_npde, inv_nobs, inv_ngh, lam_space;
  int master, pad0, pad1, pad2;
};

struct Item {
  int kind, net, begin, count, slot, face, side, pad;
};

struct Bufs {
  const float* theta;      // [n_nets][npp] canonical parameters
  const float* thetaT;     // [n_nets][nTp] transposed hidden weights W_l^T
  const NetInfo* nets;
  const float* res_pts;
  const float* obs_pts;
  const float* obs_vals;
  const float* face_pts;
  const int* face_info;    // [n_faces][3] = net_lo, net_hi, is_time
  float* nbr_val;          // [n_face_pts][2][dout]
  float* nbr_anc;          // [n_face_pts][2]
  float* nbr_res;          // interface terms: residual [n_face_pts][2][ds + 1]
  float* nbr_grd;          // and first derivatives [n_face_pts][2][dout][din]
  float* grad_part;        // [n_slots][npp]
  double* loss_part;       // [n_slots][5]
  float* stash;            // [grid][stash_per_cta]
  long long stash_per_cta;
  int* counter;            // work counter (reset before each launch)
  int* err;                // [3] error words
  int no_reverse;          // training modes: losses only, no reverse pass
  const long long* step;   // exchange: steps taken so far
  int comm_interval;       // exchange only when *step % comm_interval == 0
  const float* q_pts;      // query points [n][din]
  const int* q_perm;       // query segment order -> point index
  float* q_out;            // query output rows
  int q_w;                 // query row width
  int q_jets;              // jet queries: rows are the raw output jets [DOUT][C] (no residual, no anchoring)
};

// ------------------------------------------------------------ tiling ---
// Register tiles.  Shared memory reads at most 128 distinct bytes per clock
// per SM, against 128 FFMA per clock, so a thread tile wants about 4 FMA per
// float it loads: TM neurons x (TP points x C channels) gives
// TM*NCOL / (TM + NCOL).  W = 64 uses 8 neurons per thread (and 8 points per
// thread for values: 256-point value tiles, measured 11 % faster than 128 on
// the TGV value and exchange items); W = 128 is held to 4 neurons by the
// shared-memory capacity of its activation buffers.
// TV selects the register tile: 0 the default, 1 an alternate - at width 128
// with jets 8 neurons x 1 point per thread (the same 16-point tile, half the
// points per thread, twice the neurons), elsewhere half the points per thread
// (a tile of half the points).  The autotuner times both.
template <int W, int C, int TV = 0>
struct Tile {
  static constexpr bool WIDE_TM = (W == 64) || (W == 128 && TV == 1 && C > 1);
  static constexpr int TM = WIDE_TM ? 8 : 4;      // neurons per thread
  static constexpr int NG = W / TM;               // neuron groups
  static constexpr int PG = NT / NG;              // point groups
  static constexpr int TP0 = (W == 128) ? (C == 1 ? 8 : (C == 4 ? 4 : 2))
                           : (W == 64) ? (C == 1 ? 8 : (C == 6 ? 1 : 2))
                           : 2;
  static constexpr int TP = (TV == 0) ? TP0
                          : (W == 128 && C > 1) ? 1
                          : (TP0 == 1 ? TP0 : TP0 / 2);   // points per thread
  static constexpr int P = PG * TP;               // points per tile
  static constexpr int NCOL = TP * C;             // columns per thread
  static constexpr int PC = P * C;
  static constexpr int VEC = (NCOL % 4 == 0) ? 4 : ((NCOL % 2 == 0) ? 2 : 1);
  // Activation rows: row(i) = i*RS + SK*((i/TM) % SKM).  RS = 4 (mod 32) keeps
  // the strided rows of the weight-gradient loads on distinct banks; the skew
  // SK per neuron group separates the rows that the lanes of one
  // shared-memory phase store (8 rows apart when TM = 8).  Chosen with a
  // wavefront model of every access pattern of the kernel.
  static constexpr int RS0 = ((PC + 27) / 32) * 32 + 4;
  static constexpr int SK = WIDE_TM ? ((C == 1 || C == 4) ? 4 : 8) : 0;
  static constexpr int SKM = WIDE_TM ? ((C == 1 || C == 4) ? 2 : 4) : 1;
  static constexpr int RS = (RS0 >= PC + SK * (SKM - 1)) ? RS0 : RS0 + 32 * ((PC + SK * (SKM - 1) - RS0 + 31) / 32);
  __host__ __device__ static constexpr int row(int i) { return i * RS + SK * ((i / TM) % SKM); }
  static constexpr int NQ = TM * NCOL / 4;        // stashed float4 per thread per layer
  // weight-gradient contraction dW[i][k] = sum_pc Zb[i][pc] A[k][pc]:
  // D x D outputs per thread, K (pc) split over KS consecutive lanes
  static constexpr int D = (W >= 64) ? 8 : 4;
  static constexpr int NTI = W / D;               // tiles per matrix dimension
  static constexpr int KS = NT / (NTI * NTI);     // K-split lanes per tile
  static_assert(NG >= 8 && PG >= 4 && PG * NG == NT, "tile");
  static_assert(PC % 4 == 0 && TM % 4 == 0 && RS % 4 == 0 && SK % VEC == 0, "tile columns");
  static_assert(RS >= PC + SK * (SKM - 1), "row skew exceeds the row padding");
  static_assert(KS >= 1 && KS <= 32 && NTI * NTI * KS == NT, "weight-gradient tile");
};

template <int W, int C, int DOUT, int TV = 0>
constexpr size_t smem_floats(int L) {
  using T = Tile<W, C, TV>;
  return (size_t)2 * W * T::RS + (size_t)W * W + (size_t)2 * DOUT * T::RS + (size_t)T::P * 4 +
         (size_t)W * 4 + W + 4 + (size_t)(L > 1 ? L - 1 : 0) * W;
}

// ------------------------------------------------------- PTX helpers ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread stages `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global memory into shared memory with a bulk async copy completing on
// `bar`.  All earlier shared-memory reads of dst must be finished (a CTA
// barrier precedes every call).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of `bar`.  Bounded: after ~2 s of waiting the
// kernel records ERR_TIMEOUT and continues (its results are then invalid and
// the host reports DPINN_ERR_TIMEOUT) instead of spinning forever.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > 2000000000ull) {
      atomicExch(err + ERR_TIMEOUT, 1);
      return;
    }
  }
}

// Bounded wait for phase `parity` of `bar` (about 2 s); false on time-out.
__device__ __forceinline__ bool mbar_wait_ok(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > 2000000000ull) return false;
  }
}

// ------------------------------------------------------ jet algebra ---
// Activation jets per neuron, a = sigma(z) with s1, s2, s3 the first three
// derivatives of sigma:  d_q a = s1 d_q z,  lap a = s2 * sum_{spatial q}
// (d_q z)^2 + s1 * lap z.
//   tanh: s1 = 1 - a^2, s2 = -2 a s1, s3 = -2 s1 (1 - 3 a^2), all
//         polynomials in a, so the stash keeps a = tanh z in the value
//         channel and the reverse pass evaluates no tanh;
//   sin:  s1 = cos z, s2 = -sin z, s3 = -cos z; cos z is not a function of
//         sin z, so the stash keeps z itself.
enum { ACT_TANH = 0, ACT_SIN = 1 };

struct ActD {
  float a, s1, s2, s3;
};

// sin x and cos x for the sin activation.  Every layer of a sin network
// evaluates both at each neuron and point; the library sincosf, which serves
// arguments of any magnitude, measured 8-9 % of the streamed-weight jet
// kernels in code weight alone.  Pre-activations are O(1-10), so a
// reduction by pi/2 in three parts suffices (the Cody-Waite method, Cody and
// Waite, "Software Manual for the Elementary Functions", 1980):
// k = rint(x 2/pi), r = x - k P1 - k P2 - k P3 with P1 + P2 + P3 = pi/2 to
// 6e-18, P1 and P2 of 12 significant bits (k P1, k P2 exact for |k| < 2^12,
// |x| < 6400), each step one fused multiply-add; then the Taylor series of
// sin and cos on |r| <= pi/4, to r^9 and r^10 (truncation below 3e-9
// relative), and the quadrant k mod 4.  Within a few ulp of sin x, cos x for
// |x| < 6400 (tested against float64 through dpinn_selftest_sincos); NaN
// and inf give NaN.
__device__ __forceinline__ void sincos_act(float x, float* sn, float* cs) {
  constexpr float TWO_OVER_PI = 0x1.45f306p-1f;
  constexpr float P1 = 0x1.922p+0f, P2 = -0x1.2aep-18f, P3 = -0x1.de973ep-31f;
  const float k = rintf(x * TWO_OVER_PI);
  float r = fmaf(-k, P1, x);
  r = fmaf(-k, P2, r);
  r = fmaf(-k, P3, r);
  const float r2 = r * r;
  // sin r = r - r^3/3! + r^5/5! - r^7/7! + r^9/9!
  float ps = fmaf(r2, 1.f / 362880.f, -1.f / 5040.f);
  ps = fmaf(r2, ps, 1.f / 120.f);
  ps = fmaf(r2, ps, -1.f / 6.f);
  const float sr = fmaf(r * r2, ps, r);
  // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
  float pc = fmaf(r2, -1.f / 3628800.f, 1.f / 40320.f);
  pc = fmaf(r2, pc, -1.f / 720.f);
  pc = fmaf(r2, pc, 1.f / 24.f);
  pc = fmaf(r2, pc, -0.5f);
  const float cr = fmaf(r2, pc, 1.f);
  // x = k pi/2 + r: quadrant q = k mod 4 (two's complement keeps k < 0 right)
  const int q = static_cast<int>(k) & 3;
  const float s0 = (q & 1) ? cr : sr, c0 = (q & 1) ? sr : cr;
  *sn = (q & 2) ? -s0 : s0;
  *cs = ((q + 1) & 2) ? -c0 : c0;
}

// derivatives from the stashed value channel h0 (a for tanh, z for sin)
template <int ACT>
__device__ __forceinline__ ActD act_derivs(float h0) {
  ActD d;
  if constexpr (ACT == ACT_SIN) {
    float sn, cs;
    sincos_act(h0, &sn, &cs);
    d.a = sn; d.s1 = cs; d.s2 = -sn; d.s3 = -cs;
  } else {
    d.a = h0;
    d.s1 = 1.f - h0 * h0;
    d.s2 = -2.f * h0 * d.s1;
    d.s3 = -2.f * d.s1 * (1.f - 3.f * h0 * h0);
  }
  return d;
}

// value channel of the stashed form from the pre-activation
template <int ACT>
__device__ __forceinline__ float stash_value(float z) {
  if constexpr (ACT == ACT_SIN) return z;
  else return tanhf(z);
}

// Activation jet from the stashed form h = (h0, d_q z, lap z).
template <int C, int DS, int DIN, int ACT>
__device__ __forceinline__ void act_from_stash(const float* h, float* a) {
  if constexpr (C == 1) {
    if constexpr (ACT == ACT_SIN) {
      float c;
      sincos_act(h[0], &a[0], &c);
    } else {
      a[0] = h[0];
    }
  } else {
    const ActD d = act_derivs<ACT>(h[0]);
    a[0] = d.a;
    float S = 0.f;
#pragma unroll
    for (int q = 0; q < DS; ++q) S = fmaf(h[1 + q], h[1 + q], S);
#pragma unroll
    for (int q = 0; q < DIN; ++q) a[1 + q] = d.s1 * h[1 + q];
    a[C - 1] = fmaf(d.s2, S, d.s1 * h[C - 1]);
  }
}

// Adjoint of the activation: from the activation-jet adjoints ab to the
// pre-activation-jet adjoints zb, given the stashed form h.
template <int C, int DS, int DIN, int ACT>
__device__ __forceinline__ void act_bwd(const float* z, const float* ab, float* zb) {
  if constexpr (C == 1) {
    float s1;
    if constexpr (ACT == ACT_SIN) {
      float sn;
      sincos_act(z[0], &sn, &s1);
    }
    else s1 = 1.f - z[0] * z[0];
    zb[0] = ab[0] * s1;
  } else {
    const ActD d = act_derivs<ACT>(z[0]);
    const float al = ab[C - 1];
    float S = 0.f;
#pragma unroll
    for (int q = 0; q < DS; ++q) S = fmaf(z[1 + q], z[1 + q], S);
    float v = fmaf(ab[0], d.s1, al * fmaf(d.s3, S, d.s2 * z[C - 1]));
#pragma unroll
    for (int q = 0; q < DIN; ++q) {
      float g = ab[1 + q] * d.s1;
      if (q < DS) g = fmaf(2.f * al * d.s2, z[1 + q], g);
      zb[1 + q] = g;
      v = fmaf(ab[1 + q] * d.s2, z[1 + q], v);
    }
    zb[0] = v;
    zb[C - 1] = al * d.s1;
  }
}

// ----------------------------------------------------- smem vectors ---
template <int N, int VEC>
__device__ __forceinline__ void lds_vec(float* x, const float* p) {
  if constexpr (VEC == 4) {
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      float4 v = *reinterpret_cast<const float4*>(p + j);
      x[j] = v.x; x[j + 1] = v.y; x[j + 2] = v.z; x[j + 3] = v.w;
    }
  } else if constexpr (VEC == 2) {
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      float2 v = *reinterpret_cast<const float2*>(p + j);
      x[j] = v.x; x[j + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = p[j];
  }
}

template <int N, int VEC>
__device__ __forceinline__ void sts_vec(float* p, const float* x) {
  if constexpr (VEC == 4) {
#pragma unroll
    for (int j = 0; j < N; j += 4) *reinterpret_cast<float4*>(p + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
  } else if constexpr (VEC == 2) {
#pragma unroll
    for (int j = 0; j < N; j += 2) *reinterpret_cast<float2*>(p + j) = make_float2(x[j], x[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) p[j] = x[j];
  }
}

// acc[m][j] += sum_k Ws[k][n0 + m] * Xs[k][col0 + j],  m < TM, j < NCOL.
// Ws rows have stride ws, row k of Xs starts at rowx(k) (multiples of 4).
// The k loop is unrolled UNR deep so that the shared loads of later k steps
// issue under the FMAs of earlier ones.  Measured (jet training kernel, no
// spills at any depth): width 128 (beltrami128) 131.6 / 126.9 / 123.1 /
// 120.8 ms at depths 2 / 4 / 8 / 16; width 64 (TGV) 3.64 / 3.61 / 3.60 /
// 3.63 ms.  The kernel takes 16 at width 128 and 8 below.
template <int TM, int NCOL, int VEC, int UNR, class RowX>
__device__ __forceinline__ void contract(float (&acc)[TM][NCOL], const float* __restrict__ Ws, int ws, int n0,
                                         const float* __restrict__ Xs, RowX rowx, int col0, int K) {
#pragma unroll UNR
  for (int k = 0; k < K; ++k) {
    float w[TM];
    lds_vec<TM, 4>(w, Ws + k * ws + n0);
    float x[NCOL];
    lds_vec<NCOL, VEC>(x, Xs + rowx(k) + col0);
    if constexpr (NCOL % 2 == 0) {
      // packed dual FP32 FMA (sm_100+): two columns per instruction
#pragma unroll
      for (int m = 0; m < TM; ++m) {
        const float2 wm = make_float2(w[m], w[m]);
#pragma unroll
        for (int j = 0; j < NCOL; j += 2) {
          float2 r = __ffma2_rn(wm, make_float2(x[j], x[j + 1]), make_float2(acc[m][j], acc[m][j + 1]));
          acc[m][j] = r.x;
          acc[m][j + 1] = r.y;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int j = 0; j < NCOL; ++j) acc[m][j] = fmaf(w[m], x[j], acc[m][j]);
    }
  }
}

// contract() over the k-range [k0, k1) only.
template <int TM, int NCOL, int VEC, int UNR, class RowX>
__device__ __forceinline__ void contract_range(float (&acc)[TM][NCOL], const float* __restrict__ Ws, int ws, int n0,
                                               const float* __restrict__ Xs, RowX rowx, int col0, int k0, int k1) {
  contract<TM, NCOL, VEC, UNR>(acc, Ws + k0 * ws, ws, n0, Xs, [&](int k) { return rowx(k + k0); }, col0, k1 - k0);
}

// Deterministic block sum of one float per thread (fixed tree order).
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  }
  return s;   // valid in thread 0
}

__device__ __forceinline__ void grad_rmw(float* g, float v, bool first) {
  *g = first ? v : (*g + v);
}

// Gradient-slot accumulation: the first tile of an item stores, later ones
// add in L2 without a read-back (fire and forget).  Each address has one
// owning thread, whose operations on it stay in program order, so the sum
// order is the tile order (deterministic).
__device__ __forceinline__ void grad_acc(float* g, float v, bool first) {
  if (first) *g = v;
  else asm volatile("red.global.add.f32 [%0], %1;" ::"l"(g), "f"(v) : "memory");
}

// Navier-Stokes residuals of one point from its output jets Y[j][c]
// (c = value, d/dx_q for every input, spatial Laplacian; j = velocity
// components then pressure), Eqs. (7)-(10):
//   r_j = [d_t u_j] + sum_i u_i d_i u_j + d_j p - nu lap u_j,  r_DS = div u.
// Returns sum_j (r_j - rt_j)^2 and adds into Yb the jet adjoints of
// (sc / 2) sum_j (r_j - rt_j)^2 (residual adjoints rb_j = sc (r_j - rt_j)
// pushed through Eqs. (7)-(10)); rt = 0 when null (the PDE loss), the
// neighbour's residual for the interface residual matching.
template <int DS, int UNST, int C>
__device__ __forceinline__ void ns_residual(const float (&Y)[DS + 1][C], float nu, float (&r)[DS + 1]) {
#pragma unroll
  for (int j = 0; j < DS; ++j) {
    float v = UNST ? Y[j][1 + DS] : 0.f;
#pragma unroll
    for (int i = 0; i < DS; ++i) v = fmaf(Y[i][0], Y[j][1 + i], v);
    v += Y[DS][1 + j];
    v = fmaf(-nu, Y[j][C - 1], v);
    r[j] = v;
  }
  float dv = 0.f;
#pragma unroll
  for (int i = 0; i < DS; ++i) dv += Y[i][1 + i];
  r[DS] = dv;
}

template <int DS, int UNST, int C>
__device__ __forceinline__ float pde_seed(const float (&Y)[DS + 1][C], float nu, float sc, float (&Yb)[DS + 1][C],
                                          const float* rt = nullptr) {
  float r[DS + 1];
  ns_residual<DS, UNST, C>(Y, nu, r);
  if (rt) {
#pragma unroll
    for (int j = 0; j <= DS; ++j) r[j] -= rt[j];
  }
  float r2 = 0.f;
#pragma unroll
  for (int j = 0; j <= DS; ++j) r2 = fmaf(r[j], r[j], r2);
  float rb[DS + 1];
#pragma unroll
  for (int j = 0; j <= DS; ++j) rb[j] = sc * r[j];
#pragma unroll
  for (int j = 0; j < DS; ++j) {
    if (UNST) Yb[j][1 + DS] += rb[j];
#pragma unroll
    for (int i = 0; i < DS; ++i) {
      Yb[i][0] = fmaf(rb[j], Y[j][1 + i], Yb[i][0]);
      Yb[j][1 + i] = fmaf(rb[j], Y[i][0], Yb[j][1 + i]);
    }
    Yb[DS][1 + j] += rb[j];
    Yb[j][C - 1] = fmaf(-nu, rb[j], Yb[j][C - 1]);
  }
#pragma unroll
  for (int i = 0; i < DS; ++i) Yb[i][1 + i] += rb[DS];
  return r2;
}

// Per-point epilogue of the grouped kernels for point p (tile row sub + p of
// `item`) with output jets Y[j][c]: TRAIN returns the point's loss terms in
// l0..l3 and the output-jet adjoints in Yb; EVAL writes the neighbour
// messages; QUERY writes the output row (masters: pass 0 keeps the raw
// pressure in pkeep, pass 1 subtracts the anchor value, Eq. (15)).
template <int DS, int UNST, bool JETS, int MODE, int C>
__device__ __forceinline__ void point_epilogue(const Shape& sh, const Bufs& b, const Item& item, const NetInfo& ni,
                                               int sub, int p, bool valid, int pass, int npass, int other_master,
                                               int is_time, const float (&Y)[DS + 1][C], float (&Yb)[DS + 1][C],
                                               float& l0, float& l1, float& l2, float& l3, float& pkeep) {
  constexpr int DIN = DS + UNST;
  constexpr int DOUT = DS + 1;
  if constexpr (MODE == M_TRAIN) {
#pragma unroll
    for (int j = 0; j < DOUT; ++j)
#pragma unroll
      for (int c = 0; c < C; ++c) Yb[j][c] = 0.f;
    if constexpr (JETS) {
      if (item.kind == K_PDE) {
        const float r2 = pde_seed<DS, UNST, C>(Y, sh.nu, valid ? 2.f * sh.lam_pde * ni.inv_npde : 0.f, Yb);
        l0 = valid ? r2 : 0.f;
      } else if (valid) {   // K_FACE with the interface terms: C0 on the value channel, r and C1 matching
        const size_t pt = (size_t)(item.begin + sub + p);
        const int o = 1 - item.side;
        const float* nv = b.nbr_val + (pt * 2 + o) * DOUT;
        float su = 0.f;
#pragma unroll
        for (int c = 0; c < DS; ++c) {
          const float e = Y[c][0] - nv[c];
          su = fmaf(sh.comp_w[c] * e, e, su);
          Yb[c][0] = 2.f * sh.lam_gh_u * sh.comp_w[c] * e * ni.inv_ngh;
        }
        float Pn = nv[DS];
        if (other_master) Pn = Pn - b.nbr_anc[pt * 2 + o];   // Eq. (15)
        const float ep = Y[DS][0] - Pn;
        const float lam = is_time ? sh.lam_time : ni.lam_space;
        Yb[DS][0] = 2.f * lam * ep * ni.inv_ngh;
        l0 = su;
        l1 = ep * ep;
        const float* rt = b.nbr_res + (pt * 2 + o) * (DS + 1);
        l2 = pde_seed<DS, UNST, C>(Y, sh.nu, 2.f * sh.lam_gh_r * ni.inv_ngh, Yb, rt);
        const float* gt = b.nbr_grd + (pt * 2 + o) * DOUT * DIN;
        float sc1 = 0.f;
#pragma unroll
        for (int c = 0; c < DOUT; ++c)
#pragma unroll
          for (int q = 0; q < DIN; ++q) {
            const float e = Y[c][1 + q] - gt[c * DIN + q];
            sc1 = fmaf(e, e, sc1);
            Yb[c][1 + q] = fmaf(2.f * sh.lam_gh_c1 * ni.inv_ngh, e, Yb[c][1 + q]);
          }
        l3 = sc1;
      }
    } else if (item.kind == K_OBS) {
      float e[DS];
#pragma unroll
      for (int c = 0; c < DS; ++c) e[c] = 0.f;
      if (valid) {
        const float* ov = b.obs_vals + (size_t)(item.begin + sub + p) * DS;
#pragma unroll
        for (int c = 0; c < DS; ++c) e[c] = Y[c][0] - ov[c];
      }
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < DS; ++c) {
        s = fmaf(sh.comp_w[c] * e[c], e[c], s);
        Yb[c][0] = 2.f * sh.lam_obs * sh.comp_w[c] * e[c] * ni.inv_nobs;
      }
      l0 = s;
    } else {   // K_FACE: own side item.side, neighbour 1 - side
      float e[DS];
      float ep = 0.f;
#pragma unroll
      for (int c = 0; c < DS; ++c) e[c] = 0.f;
      if (valid) {
        const size_t pt = (size_t)(item.begin + sub + p);
        const int o = 1 - item.side;
        const float* nv = b.nbr_val + (pt * 2 + o) * DOUT;
#pragma unroll
        for (int c = 0; c < DS; ++c) e[c] = Y[c][0] - nv[c];
        float Pn = nv[DS];
        if (other_master) Pn = Pn - b.nbr_anc[pt * 2 + o];   // Eq. (15)
        ep = Y[DS][0] - Pn;
      }
      float su = 0.f;
#pragma unroll
      for (int c = 0; c < DS; ++c) {
        su = fmaf(sh.comp_w[c] * e[c], e[c], su);
        Yb[c][0] = 2.f * sh.lam_gh_u * sh.comp_w[c] * e[c] * ni.inv_ngh;
      }
      const float lam = is_time ? sh.lam_time : ni.lam_space;
      Yb[DS][0] = 2.f * lam * ep * ni.inv_ngh;
      l0 = su;
      l1 = ep * ep;
    }
  } else if constexpr (MODE == M_EVAL) {
    if (valid) {
      const size_t pt = (size_t)(item.begin + sub + p);
      if (item.kind == K_EVAL) {
#pragma unroll
        for (int j = 0; j < DOUT; ++j) b.nbr_val[(pt * 2 + item.side) * DOUT + j] = Y[j][0];
        if constexpr (JETS) {   // the interface terms' messages: residual and first derivatives
          float r[DS + 1];
          ns_residual<DS, UNST, C>(Y, sh.nu, r);
#pragma unroll
          for (int j = 0; j <= DS; ++j) b.nbr_res[(pt * 2 + item.side) * (DS + 1) + j] = r[j];
#pragma unroll
          for (int c = 0; c < DOUT; ++c)
#pragma unroll
            for (int q = 0; q < DIN; ++q)
              b.nbr_grd[((pt * 2 + item.side) * DOUT + c) * DIN + q] = Y[c][1 + q];
        }
      } else {
        b.nbr_anc[pt * 2 + item.side] = Y[DS][0];
      }
    }
  } else {   // M_QUERY
    if (valid) {
      float* o = b.q_out + (size_t)b.q_perm[item.begin + sub + p] * b.q_w;
      if (JETS && b.q_jets) {   // the net's own output jets, row [j][c] (one pass)
#pragma unroll
        for (int j = 0; j < DOUT; ++j)
#pragma unroll
          for (int c = 0; c < C; ++c) o[j * C + c] = Y[j][c];
      } else if (pass == 0) {
#pragma unroll
        for (int j = 0; j < DS; ++j) o[j] = Y[j][0];
        if (npass == 1) o[DS] = Y[DS][0] + sh.p_ref;
        else pkeep = Y[DS][0];
        if constexpr (JETS) {
#pragma unroll
          for (int j = 0; j < DS; ++j) {
            float v = UNST ? Y[j][1 + DS] : 0.f;
#pragma unroll
            for (int i = 0; i < DS; ++i) v = fmaf(Y[i][0], Y[j][1 + i], v);
            v += Y[DS][1 + j];
            v = fmaf(-sh.nu, Y[j][C - 1], v);
            o[DOUT + j] = v;
          }
          float dv = 0.f;
#pragma unroll
          for (int i = 0; i < DS; ++i) dv += Y[i][1 + i];
          o[DOUT + DS] = dv;
        }
      } else {
        o[DS] = (pkeep - Y[DS][0]) + sh.p_ref;
      }
    }
  }
}

// ------------------------------------------------------ the kernel ---
template <int W, int DS, int UNST, bool JETS, int MODE, int ACT, int TV = 0>
__global__ void __launch_bounds__(NT, 1)
    k_pinn(const Shape sh, const Bufs b, const Item* __restrict__ items, const int* __restrict__ n_items_ptr) {
  constexpr int DIN = DS + UNST;
  constexpr int C = JETS ? DIN + 2 : 1;
  constexpr int DOUT = DS + 1;
  using T = Tile<W, C, TV>;
  constexpr int P = T::P, RS = T::RS, TP = T::TP, NCOL = T::NCOL, VEC = T::VEC, PC = T::PC;
  constexpr int TM = T::TM;
  constexpr int KU = (W >= 128) ? 16 : 8;   // unroll depth of the contractions' k loops
  constexpr bool TRAIN = (MODE == M_TRAIN);

  extern __shared__ float4 sm4[];
  float* const sm = reinterpret_cast<float*>(sm4);
  float* const bufA = sm;
  float* const bufB = bufA + W * RS;
  float* const wbuf = bufB + W * RS;
  float* const ysm = wbuf + W * W;
  float* const ybsm = ysm + DOUT * RS;
  float* const xh = ybsm + DOUT * RS;   // [P][4]
  float* const w0s = xh + P * 4;        // [W][4]
  float* const b0s = w0s + W * 4;       // [W]
  float* const bLs = b0s + W;           // [4]
  float* const bls = bLs + 4;           // [L-1][W]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int s_item;
  __shared__ float s_red[NT / 32];
  __shared__ float s_scale[4];
  __shared__ int s_other_master, s_is_time;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // A quarter-warp (8 lanes) spans 2 neuron groups x 4 point groups, so the
  // 16-byte stores of a thread tile's rows (4 rows apart = 16 banks apart)
  // and columns land in 8 distinct bank groups.
  const int ng = (warp % (T::NG / 8)) * 8 + (lane >> 2);
  const int pg = (warp / (T::NG / 8)) * 4 + (lane & 3);
  const int n0 = ng * TM, p0 = pg * TP, col0 = p0 * C;
  const int L = sh.L;
  const int n_items = *n_items_ptr;
  // Algorithm 1: the messages are refreshed every I_comm iterations and the
  // cached (stale) ones are used in between.
  if (MODE == M_EVAL && b.comm_interval > 1 && (*b.step % b.comm_interval) != 0) return;
  const auto ROW = [](int i) { return T::row(i); };

  if (t == 0) mbar_init(&mbar, 1);
  __syncthreads();
  uint32_t phase = 0;
  float4* const stash = reinterpret_cast<float4*>(b.stash + (TRAIN ? (size_t)blockIdx.x * b.stash_per_cta : 0));

  // thread-tile helpers ----------------------------------------------
  auto stash_st = [&](int l, const float (&z)[TM][NCOL]) {
    const float* zf = &z[0][0];
#pragma unroll
    for (int q = 0; q < T::NQ; ++q)
      stash[((size_t)l * T::NQ + q) * NT + t] = make_float4(zf[4 * q], zf[4 * q + 1], zf[4 * q + 2], zf[4 * q + 3]);
  };
  auto stash_ld = [&](int l, float (&z)[TM][NCOL]) {
    float* zf = &z[0][0];
#pragma unroll
    for (int q = 0; q < T::NQ; ++q) {
      const float4 v = stash[((size_t)l * T::NQ + q) * NT + t];
      zf[4 * q] = v.x; zf[4 * q + 1] = v.y; zf[4 * q + 2] = v.z; zf[4 * q + 3] = v.w;
    }
  };
  // Z of the first affine map for the thread tile: z = W0 xh + b0,
  // d_q z = s_q W0[:, q], lap z = 0.
  auto layer0 = [&](float (&z)[TM][NCOL]) {
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int i = n0 + m;
#pragma unroll
      for (int pp = 0; pp < TP; ++pp) {
        const int p = p0 + pp;
        float v = b0s[i];
#pragma unroll
        for (int q = 0; q < DIN; ++q) v = fmaf(w0s[i * 4 + q], xh[p * 4 + q], v);
        z[m][pp * C] = v;
        if constexpr (JETS) {
#pragma unroll
          for (int q = 0; q < DIN; ++q) z[m][pp * C + 1 + q] = w0s[i * 4 + q] * s_scale[q];
          z[m][pp * C + C - 1] = 0.f;
        }
      }
    }
  };
  // z -> stashed form in place (value channel: tanh z, or z for sin)
  auto to_stash_form = [&](float (&z)[TM][NCOL]) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int pp = 0; pp < TP; ++pp) z[m][pp * C] = stash_value<ACT>(z[m][pp * C]);
  };
  // activations of the thread tile (from the stashed form) into smem
  auto act_store = [&](float* buf, const float (&h)[TM][NCOL]) {
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      float a[NCOL];
#pragma unroll
      for (int pp = 0; pp < TP; ++pp) act_from_stash<C, DS, DIN, ACT>(&h[m][pp * C], &a[pp * C]);
      sts_vec<NCOL, VEC>(buf + ROW(n0 + m) + col0, a);
    }
  };

  for (;;) {
    if (t == 0) s_item = atomicAdd(b.counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const Item item = items[it];
    const int net = item.net;
    const float* const th = b.theta + (size_t)net * sh.npp;
    const float* const thT = b.thetaT + (size_t)net * sh.nTp;
    const NetInfo ni = b.nets[net];
    for (int e = t; e < W * DIN; e += NT) w0s[(e / DIN) * 4 + e % DIN] = th[sh.woff[0] + e];
    for (int e = t; e < W; e += NT) b0s[e] = th[sh.boff[0] + e];
    for (int e = t; e < (L - 1) * W; e += NT) bls[e] = th[sh.boff[1 + e / W] + e % W];
    if (t < DOUT) bLs[t] = th[sh.boff[L] + t];
    // scale from global memory: a run-time index into the local copy ni would
    // move that copy to the stack
    if (t < 4) s_scale[t] = t < DIN ? b.nets[net].scale[t] : 0.f;
    if (t == 0) {
      if (item.kind == K_FACE) {
        const int other = b.face_info[item.face * 3 + (1 - item.side)];
        s_other_master = b.nets[other].master;
        s_is_time = b.face_info[item.face * 3 + 2];
      } else {
        s_other_master = 0;
        s_is_time = 0;
      }
    }
    double lsum0 = 0.0, lsum1 = 0.0, lsum2 = 0.0, lsum3 = 0.0;   // thread 0: loss numerators of this item
    const int npass = (MODE == M_QUERY && ni.master && !b.q_jets) ? 2 : 1;

    for (int sub = 0; sub < item.count; sub += P) {
      const int npts = min(P, item.count - sub);
      const bool first = (sub == 0);
      float pkeep = 0.f;   // query: raw pressure of a master point (thread t = point)
      float* cur = bufA;   // holds A_{L-1} after the forward
      float* oth = bufB;
      for (int pass = 0; pass < npass; ++pass) {
        // ---- inputs mapped to the net's box: xh = (x - c) * s
        if (t < P) {
          float x[4] = {0.f, 0.f, 0.f, 0.f};
          const bool valid = t < npts;
          if (valid) {
            const float* src;
            if (MODE == M_QUERY) src = b.q_pts + (size_t)b.q_perm[item.begin + sub + t] * DIN;
            else if (item.kind == K_PDE) src = b.res_pts + (size_t)(item.begin + sub + t) * DIN;
            else if (item.kind == K_OBS) src = b.obs_pts + (size_t)(item.begin + sub + t) * DIN;
            else src = b.face_pts + (size_t)(item.begin + sub + t) * DIN;
#pragma unroll
            for (int q = 0; q < DIN; ++q) x[q] = src[q];
            if (pass == 1 || item.kind == K_EVAL_ANC) {
#pragma unroll
              for (int q = 0; q < DS; ++q) x[q] = sh.anchor[q];
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) xh[t * 4 + q] = (valid && q < DIN) ? (x[q] - ni.center[q]) * ni.scale[q] : 0.f;
        }
        __syncthreads();
        if (t == 0) {
          if (L >= 2) bulk_load(wbuf, thT, W * W * 4, &mbar);
          else bulk_load(wbuf, th + sh.woff[L], DOUT * W * 4, &mbar);
        }
        // ---- forward
        {
          float z[TM][NCOL];
          layer0(z);
          to_stash_form(z);
          if (TRAIN) stash_st(0, z);
          act_store(bufA, z);
        }
        cur = bufA;
        oth = bufB;
        for (int l = 1; l < L; ++l) {
          mbar_wait(&mbar, phase & 1, b.err);
          ++phase;
          __syncthreads();
          float z[TM][NCOL];
#pragma unroll
          for (int m = 0; m < TM; ++m)
#pragma unroll
            for (int j = 0; j < NCOL; ++j) z[m][j] = 0.f;
          contract<TM, NCOL, VEC, KU>(z, wbuf, W, n0, cur, ROW, col0, W);
#pragma unroll
          for (int m = 0; m < TM; ++m)
#pragma unroll
            for (int pp = 0; pp < TP; ++pp) z[m][pp * C] += bls[(l - 1) * W + n0 + m];
          __syncthreads();
          if (t == 0) {
            if (l + 1 < L) bulk_load(wbuf, thT + (size_t)l * W * W, W * W * 4, &mbar);
            else bulk_load(wbuf, th + sh.woff[L], DOUT * W * 4, &mbar);
          }
          to_stash_form(z);
          if (TRAIN) stash_st(l, z);
          act_store(oth, z);
          float* tmp = cur; cur = oth; oth = tmp;
        }
        // ---- output layer: Y[j][p][c] = W_L[j] . A[.][p][c] (+ b_L on values)
        mbar_wait(&mbar, phase & 1, b.err);
        ++phase;
        __syncthreads();
        {
          constexpr int PAIRS = DOUT * P;
          constexpr int KS0 = NT / PAIRS;
          constexpr int KS = KS0 >= 4 ? 4 : (KS0 >= 2 ? 2 : 1);
          for (int pr = t / KS; pr < PAIRS; pr += NT / KS) {
            const int j = pr / P, p = pr % P, lk = t % KS;
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = 0.f;
            for (int k = lk; k < W; k += KS) {
              const float w = wbuf[j * W + k];
#pragma unroll
              for (int c = 0; c < C; ++c) acc[c] = fmaf(w, cur[ROW(k) + p * C + c], acc[c]);
            }
#pragma unroll
            for (int o = KS / 2; o > 0; o >>= 1)
#pragma unroll
              for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
            if (lk == 0) {
#pragma unroll
              for (int c = 0; c < C; ++c) ysm[j * RS + p * C + c] = acc[c] + (c == 0 ? bLs[j] : 0.f);
            }
          }
        }
        __syncthreads();
        // ---- per-point epilogue
        float l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;
        if (t < P) {
          const int p = t;
          const bool valid = p < npts;
          float Y[DOUT][C];
#pragma unroll
          for (int j = 0; j < DOUT; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) Y[j][c] = ysm[j * RS + p * C + c];
          float Yb[DOUT][C];
          point_epilogue<DS, UNST, JETS, MODE, C>(sh, b, item, ni, sub, p, valid, pass, npass, s_other_master,
                                                  s_is_time, Y, Yb, l0, l1, l2, l3, pkeep);
          if constexpr (MODE == M_TRAIN) {
#pragma unroll
            for (int j = 0; j < DOUT; ++j)
#pragma unroll
              for (int c = 0; c < C; ++c) ybsm[j * RS + p * C + c] = Yb[j][c];
          }
        }
        if constexpr (TRAIN) {
          const float s0 = block_sum(l0, s_red);
          if (t == 0) lsum0 += (double)s0;
          if (item.kind == K_FACE) {
            const float s1 = block_sum(l1, s_red);
            if (t == 0) lsum1 += (double)s1;
            if constexpr (JETS) {
              const float s2 = block_sum(l2, s_red);
              if (t == 0) lsum2 += (double)s2;
              const float s3 = block_sum(l3, s_red);
              if (t == 0) lsum3 += (double)s3;
            }
          }
        }
        __syncthreads();
      }   // pass
      if constexpr (!TRAIN) continue;
      if (b.no_reverse) continue;

      // ================= reverse pass =================
      float* const g = b.grad_part + (size_t)item.slot * sh.npp;
      // output layer: dW_L, db_L, and A_{L-1} adjoints
      for (int e = t; e < DOUT * W; e += NT) {
        const int j = e / W, k = e % W;
        float s = 0.f;
        for (int pc = 0; pc < PC; ++pc) s = fmaf(ybsm[j * RS + pc], cur[ROW(k) + pc], s);
        grad_rmw(g + sh.woff[L] + e, s, first);
      }
      if (t < DOUT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += ybsm[t * RS + p * C];
        grad_rmw(g + sh.boff[L] + t, s, first);
      }
      float* zb = oth;
      float* ab = cur;
      {
        float a[TM][NCOL];
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int j = 0; j < NCOL; ++j) a[m][j] = 0.f;
        contract<TM, NCOL, VEC, KU>(a, wbuf, W, n0, ybsm, ROW, col0, DOUT);
        __syncthreads();
        if (t == 0 && L >= 2) bulk_load(wbuf, th + sh.woff[L - 1], W * W * 4, &mbar);
        float z[TM][NCOL];
        stash_ld(L - 1, z);
#pragma unroll
        for (int m = 0; m < TM; ++m) {
          float zz[NCOL];
#pragma unroll
          for (int pp = 0; pp < TP; ++pp) act_bwd<C, DS, DIN, ACT>(&z[m][pp * C], &a[m][pp * C], &zz[pp * C]);
          sts_vec<NCOL, VEC>(zb + ROW(n0 + m) + col0, zz);
        }
      }
      for (int l = L - 1; l >= 1; --l) {
        __syncthreads();
        {   // A_{l-1} into ab
          float z[TM][NCOL];
          stash_ld(l - 1, z);
          act_store(ab, z);
        }
        __syncthreads();
        // dW_l[i][k] += sum_pc Zb_l[i][pc] A_{l-1}[k][pc].  Tile (ig, kg) owns
        // rows ig + NTI a and columns kg + NTI c; its KS lanes take interleaved
        // float4 chunks of pc.  The lanes' partial tiles are combined by a
        // shuffle reduce-scatter in a fixed order (lane ks ends with flat
        // entries [NE ks, NE ks + NE) of the tile), which go into the item's
        // gradient slot between the chunks of the next contraction: stored by
        // the item's first tile, added by later ones with L2 reductions (no
        // read-back).  With KS > 1 the chunk offset moves the bank group, so kg
        // is permuted to keep a quarter-warp's rows 4 groups apart.
        constexpr int D = T::D, NTI = T::NTI, KS = T::KS, NE = D * D / KS;
        const int ks = t % KS, tile = t / KS;
        const int kq = tile % NTI;
        const int kg = (KS > 1 && NTI == 8) ? ((kq & 1) * 4 + (kq >> 1)) : kq;
        const int ig = tile / NTI;
        float dwv[NE];
        {
          float2 acc2[D][D];
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) acc2[a][c] = make_float2(0.f, 0.f);
          for (int pc = 4 * ks; pc < PC; pc += 4 * KS) {
            float4 zv[D], av[D];
#pragma unroll
            for (int a = 0; a < D; ++a) zv[a] = *reinterpret_cast<const float4*>(zb + ROW(ig + NTI * a) + pc);
#pragma unroll
            for (int c = 0; c < D; ++c) av[c] = *reinterpret_cast<const float4*>(ab + ROW(kg + NTI * c) + pc);
            // packed dual FMA: lane .x sums the even, .y the odd pc of a chunk
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int c = 0; c < D; ++c) {
                float2 s = acc2[a][c];
                s = __ffma2_rn(make_float2(zv[a].x, zv[a].y), make_float2(av[c].x, av[c].y), s);
                s = __ffma2_rn(make_float2(zv[a].z, zv[a].w), make_float2(av[c].z, av[c].w), s);
                acc2[a][c] = s;
              }
          }
          float v[D * D];
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) v[a * D + c] = acc2[a][c].x + acc2[a][c].y;
          // reduce-scatter over the KS lanes of the tile: at offset o the
          // lane keeps the half selected by bit o of ks and adds the partner's
#pragma unroll
          for (int o = KS / 2, S = D * D; o > 0; o >>= 1, S >>= 1) {
            const bool hi = (ks & o) != 0;
#pragma unroll
            for (int i = 0; i < S / 2; ++i) {
              const float send = hi ? v[i] : v[i + S / 2];
              const float keep = hi ? v[i + S / 2] : v[i];
              v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
#pragma unroll
          for (int i = 0; i < NE; ++i) dwv[i] = v[i];
        }
        for (int e = t; e < W; e += NT) {
          float s = 0.f;
          for (int p = 0; p < P; ++p) s += zb[ROW(e) + p * C];
          grad_rmw(g + sh.boff[l] + e, s, first);
        }
        float* const gw = g + sh.woff[l];
        const auto waddr = [&](int i) {
          const int e = NE * ks + i;
          return gw + (ig + NTI * (e / D)) * W + kg + NTI * (e % D);
        };
        // A_{l-1} adjoint = W_l^T Zb_l; the dW entries go out between its
        // chunks (stores for the item's first tile, then L2 reductions)
        mbar_wait(&mbar, phase & 1, b.err);
        ++phase;
        float a[TM][NCOL];
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int j = 0; j < NCOL; ++j) a[m][j] = 0.f;
        {
          constexpr int NCH = 8, NEH = (NE + NCH - 1) / NCH;
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            contract_range<TM, NCOL, VEC, KU>(a, wbuf, W, n0, zb, ROW, col0, ch * (W / NCH), (ch + 1) * (W / NCH));
#pragma unroll
            for (int q = 0; q < NEH; ++q) {
              const int i = ch * NEH + q;
              if (i < NE) grad_acc(waddr(i), dwv[i], first);
            }
          }
        }
        __syncthreads();
        if (t == 0 && l - 1 >= 1) bulk_load(wbuf, th + sh.woff[l - 1], W * W * 4, &mbar);
        float z[TM][NCOL];
        stash_ld(l - 1, z);
#pragma unroll
        for (int m = 0; m < TM; ++m) {
          float zz[NCOL];
#pragma unroll
          for (int pp = 0; pp < TP; ++pp) act_bwd<C, DS, DIN, ACT>(&z[m][pp * C], &a[m][pp * C], &zz[pp * C]);
          sts_vec<NCOL, VEC>(zb + ROW(n0 + m) + col0, zz);
        }
      }
      __syncthreads();
      // first affine map: dW_0[i][q] += sum_p (Zb_val xh_q + s_q Zb_q), db_0
      for (int e = t; e < W * DIN; e += NT) {
        const int i = e / DIN, q = e % DIN;
        float s = 0.f;
        for (int p = 0; p < P; ++p) {
          s = fmaf(zb[ROW(i) + p * C], xh[p * 4 + q], s);
          if constexpr (JETS) s = fmaf(s_scale[q], zb[ROW(i) + p * C + 1 + q], s);
        }
        grad_rmw(g + sh.woff[0] + e, s, first);
      }
      for (int e = t; e < W; e += NT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += zb[ROW(e) + p * C];
        grad_rmw(g + sh.boff[0] + e, s, first);
      }
      __syncthreads();
    }   // sub-tiles
    if (TRAIN && t == 0) {
      double* lp = b.loss_part + (size_t)item.slot * LP;
      for (int q = 0; q < LP; ++q) lp[q] = 0.0;
      if (item.kind == K_PDE) lp[1] = lsum0;
      else if (item.kind == K_OBS) lp[0] = lsum0;
      else {
        lp[2] = lsum0;
        lp[s_is_time ? 4 : 3] = lsum1;
        lp[5] = lsum2;
        lp[6] = lsum3;
      }
    }
  }   // items
}

}  // namespace dk

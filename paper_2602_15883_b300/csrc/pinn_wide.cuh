// Grouped kernel for the widths that the register-tiled kernel does not
// tile: the cylinder networks of Sec. 5 (6 x 150 and 8 x 200 neurons).  It
// computes exactly what k_pinn computes (Eqs. (5)-(16), Algorithm 1; the
// per-point epilogue is the same function), with a layout that takes any
// width W <= WP (WP a multiple of 32):
//   * lane l of every warp owns neurons l, l + 32, ... (TMG = WP / 32 of them)
//     and warp w owns the tile's points w TPG ... w TPG + TPG - 1 (its column
//     group), so the activation jets of a (neuron, point) stay in one thread;
//   * a W x W weight matrix does not fit in shared memory next to the
//     activations (200 x 200 fp32 = 160 KB), so it is streamed through two
//     buffers of 32 rows (16 above width 160), the next chunk arriving while
//     the previous one is contracted.  The streamed copies (W_l^T for the
//     forward product, W_l for the adjoint one) are kept per step in a
//     padded, lane-blocked column order (wide_pos): a chunk is one
//     contiguous block, moved by one bulk asynchronous copy (the copy
//     engine, not the threads) completing on the buffer's mbarrier, and a
//     lane reads its TMG weights of a row with float4 / float2 loads;
//   * the weight gradient is accumulated per block of 5-8 output neurons
//     per warp (sized so that no block pads a row beyond the width) and added
//     to the item's slot with coalesced L2 reductions (lanes = input
//     neurons).
// Rows of the activation buffers are 4 (mod 32) floats apart when a warp's
// columns come in 4-aligned groups (16-byte column accesses), else 2 (mod
// 32): either way the lane-strided row accesses of the weight gradient and
// of the activation stores are conflict-free.
#pragma once
#include "pinn_kernels.cuh"

namespace dk {

constexpr int NTW = 256;   // threads per CTA of the wide kernel
template <int N> struct IntC { static constexpr int value = N; };   // a block size as a type
static_assert(NTW == NT, "the block sums and launches assume NT threads");

// TV selects the register tile: 0 the default (2 points per warp with jets,
// 8 with values), 1 an alternate with half of that (1 and 4); the autotuner
// times both.
template <int WP, int C, int TV = 0>
struct WideTile {
  static_assert(WP % 32 == 0, "padded width");
  static constexpr int TMG = WP / 32;                                              // neurons per thread
  static constexpr int TPG = (C == 1) ? (TV ? 4 : 8) : (TV ? 1 : 2);             // points per column group
  static constexpr int P = 8 * TPG;                                                // points per tile
  static constexpr int NCOL = TPG * C;                                             // columns per thread
  static constexpr int PC = P * C;
  // 16-byte column accesses when a warp's columns are 4-aligned; the row
  // stride is then 4 (mod 32), else 2 (mod 32), so that lane-strided rows
  // (32 rows RS apart) read or written 16 (else 8) bytes per lane are
  // conflict-free
  static constexpr bool V4 = (NCOL % 4 == 0);
  static constexpr int RS = V4 ? ((PC + 27) / 32) * 32 + 4 : ((PC + 29) / 32) * 32 + 2;   // row stride
  static constexpr int KC = (WP > 160) ? 16 : 32;                                 // streamed weight rows
  static constexpr int NQ = TMG * NCOL;                                            // stashed floats per thread
  static constexpr uint32_t STASH_LAYER_BYTES = (uint32_t)NQ * NTW * 4;           // one layer of a CTA's stash
  static_assert(RS >= PC && RS % 2 == 0 && P <= NTW && PC % 4 == 0, "wide tile");
  static_assert(STASH_LAYER_BYTES % 128 == 0, "stash blocks are whole 128-byte lines");
};

template <int WP, int C, int DOUT, int TV = 0>
constexpr size_t smem_floats_wide(int L) {
  using T = WideTile<WP, C, TV>;
  return (size_t)2 * WP * T::RS + (size_t)2 * T::KC * WP + (size_t)2 * DOUT * T::RS + (size_t)T::P * 4 +
         (size_t)WP * 4 + WP + 4 + (size_t)(L > 1 ? L - 1 : 0) * WP;
}

// L2 residency of the stash: a block is prefetched into L2 (one bulk
// prefetch, two reverse layers ahead of its reads) and discarded from L2
// after its last read (no write-back of dead lines).
__device__ __forceinline__ void wide_l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void wide_l2_discard(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Streaming state of the two weight-chunk buffers.  Buffer b's copies
// complete on bar[b], one copy outstanding at most (a copy into b is issued
// only after every thread has waited for b's previous one).  A wait that
// runs out (about 2 s) records ERR_TIMEOUT and sets *abort: no later copy is
// issued and no later wait taken, so the kernel ends (with invalid results,
// which the host reports) instead of spinning.
struct WStream {
  uint64_t* bar;                // [2] shared: copy completion per buffer
  int* abort;                   // shared
  int* err;                     // global error words
  uint32_t waited0, waited1;    // per thread: copies of buffer 0 / 1 waited for
  uint32_t issued0, issued1;    // thread 0: copies issued into buffer 0 / 1
};
// (scalar pairs, not arrays: a run-time buffer index into an array member
// would move the whole struct to the stack)

// Rows [r0, r0 + nr) of a streamed-weight block (rows of WP floats, 16-byte
// aligned, contiguous) into buffer b: one bulk copy by thread 0.  Every
// earlier read of the buffer precedes a CTA barrier before the call.
template <int WP>
__device__ __forceinline__ void wide_chunk_issue(WStream& ws, int b, float* dst, const float* __restrict__ src, int r0,
                                                 int nr) {
  static_assert(WP % 4 == 0, "16-byte rows");
  if (threadIdx.x == 0 && !*(volatile int*)ws.abort) {
    bulk_load(dst, src + (size_t)r0 * WP, (uint32_t)(nr * WP * 4), &ws.bar[b]);
    if (b) ++ws.issued1;
    else ++ws.issued0;
  }
}
__device__ __forceinline__ void wide_chunk_wait(WStream& ws, int b) {
  const uint32_t n = b ? ws.waited1 : ws.waited0;
  if (!*(volatile int*)ws.abort && !mbar_wait_ok(&ws.bar[b], n & 1)) {
    *ws.abort = 1;
    atomicExch(ws.err + ERR_TIMEOUT, 1);
  }
  if (b) ++ws.waited1;
  else ++ws.waited0;
}

// The weights of row k of a streamed chunk for the thread's neurons
// lane + 32 m (the lane-blocked order of wide_pos): float4 groups, then a
// float2 pair and a single entry as the width requires.
template <int WP>
__device__ __forceinline__ void wide_row_weights(const float* row, int lane, float (&w)[WP / 32]) {
  constexpr int TMG = WP / 32, G4 = TMG / 4, REM = TMG - 4 * G4;
#pragma unroll
  for (int a = 0; a < G4; ++a) {
    const float4 v = *reinterpret_cast<const float4*>(row + a * 128 + lane * 4);
    w[4 * a] = v.x; w[4 * a + 1] = v.y; w[4 * a + 2] = v.z; w[4 * a + 3] = v.w;
  }
  if constexpr (REM >= 2) {
    const float2 v = *reinterpret_cast<const float2*>(row + G4 * 128 + lane * 2);
    w[4 * G4] = v.x; w[4 * G4 + 1] = v.y;
  }
  if constexpr (REM % 2 == 1) w[TMG - 1] = row[G4 * 128 + (REM >= 2 ? 64 : 0) + lane];
}

// acc[m][j] += sum_{k < K} M[k][lane + 32 m] * X[k * RS + col0 + j], M a
// K x WP block of the streamed-weight layout (wide_pos column order, padded
// neurons zero) in global memory, streamed in chunks of KC rows through two
// buffers.  One barrier per chunk, after the wait for its copy: it shows
// that every warp has finished chunk ch - 1, whose buffer then takes chunk
// ch + 1 while chunk ch is contracted.  (A second loop of compile-time
// length for full chunks measured 1-5 % slower in this kernel: code size.)
// Ends with a barrier (the buffers and X may be rewritten afterwards).
template <int WP, int C, int NCOL, int TV>
__device__ __forceinline__ void wide_contract(float (&acc)[WP / 32][NCOL], const float* __restrict__ M, int K,
                                              float* wch, const float* X, int col0, WStream& ws) {
  using T = WideTile<WP, C, TV>;
  constexpr int KC = T::KC, TMG = T::TMG, RS = T::RS;
  const int lane = threadIdx.x & 31;
  const int nch = (K + KC - 1) / KC;
  wide_chunk_issue<WP>(ws, 0, wch, M, 0, min(KC, K));
  for (int ch = 0; ch < nch; ++ch) {
    float* const buf = wch + (ch & 1) * KC * WP;
    wide_chunk_wait(ws, ch & 1);
    __syncthreads();
    if (ch + 1 < nch)
      wide_chunk_issue<WP>(ws, (ch + 1) & 1, wch + ((ch + 1) & 1) * KC * WP, M, (ch + 1) * KC,
                           min(KC, K - (ch + 1) * KC));
    const int k0 = ch * KC, nk = min(KC, K - k0);
    auto row = [&](int k) {
      float w[TMG];
      wide_row_weights<WP>(buf + k * WP, lane, w);
      const float* xr = X + (k0 + k) * RS + col0;
      if constexpr (T::V4) {
#pragma unroll
        for (int j = 0; j < NCOL; j += 4) {
          const float4 x = *reinterpret_cast<const float4*>(xr + j);
#pragma unroll
          for (int m = 0; m < TMG; ++m) {
            const float2 r0 = __ffma2_rn(make_float2(w[m], w[m]), make_float2(x.x, x.y),
                                         make_float2(acc[m][j], acc[m][j + 1]));
            const float2 r1 = __ffma2_rn(make_float2(w[m], w[m]), make_float2(x.z, x.w),
                                         make_float2(acc[m][j + 2], acc[m][j + 3]));
            acc[m][j] = r0.x;
            acc[m][j + 1] = r0.y;
            acc[m][j + 2] = r1.x;
            acc[m][j + 3] = r1.y;
          }
        }
      } else if constexpr (NCOL % 2 == 0) {
#pragma unroll
        for (int j = 0; j < NCOL; j += 2) {
          const float2 x = *reinterpret_cast<const float2*>(xr + j);
#pragma unroll
          for (int m = 0; m < TMG; ++m) {
            const float2 r = __ffma2_rn(make_float2(w[m], w[m]), x, make_float2(acc[m][j], acc[m][j + 1]));
            acc[m][j] = r.x;
            acc[m][j + 1] = r.y;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          const float x = xr[j];
#pragma unroll
          for (int m = 0; m < TMG; ++m) acc[m][j] = fmaf(w[m], x, acc[m][j]);
        }
      }
    };
    // unrolled 8 deep (measured: at width 224, 16 deep +0.2 %; at width 160,
    // 4 deep 1.3 % slower once the sin evaluation and stack frames were gone)
    constexpr int UNR = 8;
#pragma unroll UNR
    for (int k = 0; k < nk; ++k) row(k);
  }
  __syncthreads();
}

template <int WP, int DS, int UNST, bool JETS, int MODE, int ACT, int TV = 0>
__global__ void __launch_bounds__(NTW, 1)
    k_pinn_w(const Shape sh, const Bufs b, const Item* __restrict__ items, const int* __restrict__ n_items_ptr) {
  constexpr int DIN = DS + UNST;
  constexpr int C = JETS ? DIN + 2 : 1;
  constexpr int DOUT = DS + 1;
  using T = WideTile<WP, C, TV>;
  constexpr int P = T::P, RS = T::RS, TPG = T::TPG, NCOL = T::NCOL, PC = T::PC, TMG = T::TMG, KC = T::KC;
  constexpr bool TRAIN = (MODE == M_TRAIN);

  extern __shared__ float4 sm4[];
  float* const sm = reinterpret_cast<float*>(sm4);
  float* const bufA = sm;
  float* const bufB = bufA + WP * RS;
  float* const wch = bufB + WP * RS;        // [2][KC][WP]
  float* const ysm = wch + 2 * KC * WP;
  float* const ybsm = ysm + DOUT * RS;
  float* const xh = ybsm + DOUT * RS;       // [P][4]
  float* const w0s = xh + P * 4;            // [WP][4]
  float* const b0s = w0s + WP * 4;          // [WP]
  float* const bLs = b0s + WP;              // [4]
  float* const bls = bLs + 4;               // [L-1][WP]
  __shared__ int s_item;
  __shared__ float s_red[NTW / 32];
  __shared__ float s_scale[4];
  __shared__ int s_other_master, s_is_time;
  __shared__ __align__(8) uint64_t s_wbar[2];   // weight-chunk copies
  __shared__ int s_wabort;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int W = sh.W, L = sh.L;
  const int col0 = warp * NCOL;             // the warp's points warp * TPG + [0, TPG)
  const int n_items = *n_items_ptr;
  if (MODE == M_EVAL && b.comm_interval > 1 && (*b.step % b.comm_interval) != 0) return;

  if (t == 0) {
    mbar_init(&s_wbar[0], 1);
    mbar_init(&s_wbar[1], 1);
    s_wabort = 0;
  }
  WStream ws{s_wbar, &s_wabort, b.err, 0u, 0u, 0u, 0u};
  // padded neurons (>= W) see zero weights (the streamed layout holds zeros
  // there) and zero biases, so every value stays finite
  for (int e = t; e < WP * 4; e += NTW) w0s[e] = 0.f;
  for (int e = t; e < WP; e += NTW) b0s[e] = 0.f;
  for (int e = t; e < (L - 1) * WP; e += NTW) bls[e] = 0.f;
  __syncthreads();
  float* const stash = b.stash + (TRAIN ? (size_t)blockIdx.x * b.stash_per_cta : 0);

  auto stash_st = [&](int l, const float (&z)[TMG][NCOL]) {
#pragma unroll
    for (int m = 0; m < TMG; ++m)
#pragma unroll
      for (int j = 0; j < NCOL; ++j) stash[((size_t)l * T::NQ + m * NCOL + j) * NTW + t] = z[m][j];
  };
  auto stash_ld = [&](int l, float (&z)[TMG][NCOL]) {
#pragma unroll
    for (int m = 0; m < TMG; ++m)
#pragma unroll
      for (int j = 0; j < NCOL; ++j) z[m][j] = stash[((size_t)l * T::NQ + m * NCOL + j) * NTW + t];
  };
  auto to_stash_form = [&](float (&z)[TMG][NCOL]) {
#pragma unroll
    for (int m = 0; m < TMG; ++m)
#pragma unroll
      for (int pp = 0; pp < TPG; ++pp) z[m][pp * C] = stash_value<ACT>(z[m][pp * C]);
  };
  // the thread's NCOL columns of neuron lane + 32 m -> its row of buf
  auto row_store = [&](float* buf, int m, const float (&a)[NCOL]) {
    float* row = buf + (lane + 32 * m) * RS + col0;
    if constexpr (T::V4) {
#pragma unroll
      for (int j = 0; j < NCOL; j += 4) *reinterpret_cast<float4*>(row + j) = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < NCOL; ++j) row[j] = a[j];
    }
  };
  auto act_store = [&](float* buf, const float (&h)[TMG][NCOL]) {
#pragma unroll
    for (int m = 0; m < TMG; ++m) {
      float a[NCOL];
#pragma unroll
      for (int pp = 0; pp < TPG; ++pp) act_from_stash<C, DS, DIN, ACT>(&h[m][pp * C], &a[pp * C]);
      row_store(buf, m, a);
    }
  };
  auto stash_prefetch = [&](int l) {
    if (t == 0) wide_l2_prefetch(stash + (size_t)l * T::NQ * NTW, T::STASH_LAYER_BYTES);
  };
  auto stash_discard = [&](int l) {   // after a barrier that follows the block's last reads
    for (uint32_t o = (uint32_t)t * 128; o < T::STASH_LAYER_BYTES; o += NTW * 128)
      wide_l2_discard(reinterpret_cast<const char*>(stash + (size_t)l * T::NQ * NTW) + o);
  };
  auto zero_acc = [&](float (&z)[TMG][NCOL]) {
#pragma unroll
    for (int m = 0; m < TMG; ++m)
#pragma unroll
      for (int j = 0; j < NCOL; ++j) z[m][j] = 0.f;
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
    for (int e = t; e < W * DIN; e += NTW) w0s[(e / DIN) * 4 + e % DIN] = th[sh.woff[0] + e];
    for (int e = t; e < W; e += NTW) b0s[e] = th[sh.boff[0] + e];
    for (int e = t; e < (L - 1) * W; e += NTW) bls[(e / W) * WP + e % W] = th[sh.boff[1 + e / W] + e % W];
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
    double lsum0 = 0.0, lsum1 = 0.0, lsum2 = 0.0, lsum3 = 0.0;
    const int npass = (MODE == M_QUERY && ni.master && !b.q_jets) ? 2 : 1;

    for (int sub = 0; sub < item.count; sub += P) {
      const int npts = min(P, item.count - sub);
      const bool first = (sub == 0);
      float pkeep = 0.f;
      float* cur = bufA;
      float* oth = bufB;
      for (int pass = 0; pass < npass; ++pass) {
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
        // ---- first affine map: z = W0 xh + b0, d_q z = s_q W0[:, q], lap z = 0
        {
          float z[TMG][NCOL];
#pragma unroll
          for (int m = 0; m < TMG; ++m) {
            const int i = lane + 32 * m;
#pragma unroll
            for (int pp = 0; pp < TPG; ++pp) {
              const int p = warp * TPG + pp;
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
          to_stash_form(z);
          if (TRAIN) stash_st(0, z);
          act_store(bufA, z);
        }
        cur = bufA;
        oth = bufB;
        // ---- hidden layers (the contraction's first barrier orders the stores above)
        for (int l = 1; l < L; ++l) {
          float z[TMG][NCOL];
          zero_acc(z);
          wide_contract<WP, C, NCOL, TV>(z, thT + (size_t)(l - 1) * 2 * W * WP, W, wch, cur, col0, ws);
#pragma unroll
          for (int m = 0; m < TMG; ++m)
#pragma unroll
            for (int pp = 0; pp < TPG; ++pp) z[m][pp * C] += bls[(l - 1) * WP + lane + 32 * m];
          to_stash_form(z);
          if (TRAIN) stash_st(l, z);
          act_store(oth, z);
          float* tmp = cur; cur = oth; oth = tmp;
        }
        __syncthreads();
        // ---- output layer: Y[j][p][c] = W_L[j] . A[.][p][c] (+ b_L on values)
        {
          const float* const wL = th + sh.woff[L];
          constexpr int PAIRS = DOUT * P;
          constexpr int KS0 = NTW / PAIRS;
          constexpr int KS = KS0 >= 8 ? 8 : (KS0 >= 4 ? 4 : (KS0 >= 2 ? 2 : 1));
          for (int pr = t / KS; pr < PAIRS; pr += NTW / KS) {
            const int j = pr / P, p = pr % P, lk = t % KS;
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = 0.f;
            for (int k = lk; k < W; k += KS) {
              const float w = wL[j * W + k];
#pragma unroll
              for (int c = 0; c < C; ++c) acc[c] = fmaf(w, cur[k * RS + p * C + c], acc[c]);
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
      // output layer: dW_L, db_L
      for (int e = t; e < DOUT * W; e += NTW) {
        const int j = e / W, k = e % W;
        float s = 0.f;
        for (int pc = 0; pc < PC; ++pc) s = fmaf(ybsm[j * RS + pc], cur[k * RS + pc], s);
        grad_acc(g + sh.woff[L] + e, s, first);
      }
      if (t < DOUT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += ybsm[t * RS + p * C];
        grad_acc(g + sh.boff[L] + t, s, first);
      }
      float* zb = oth;
      float* ab = cur;
      {   // A_{L-1} adjoints = W_L^T Yb, then through the activation
        const float* const wL = th + sh.woff[L];
        float a[TMG][NCOL];
        zero_acc(a);
#pragma unroll
        for (int jo = 0; jo < DOUT; ++jo) {
          float yb[NCOL];
#pragma unroll
          for (int j = 0; j < NCOL; ++j) yb[j] = ybsm[jo * RS + col0 + j];
#pragma unroll
          for (int m = 0; m < TMG; ++m) {
            const int k = lane + 32 * m;
            const float w = k < W ? wL[jo * W + k] : 0.f;
#pragma unroll
            for (int j = 0; j < NCOL; ++j) a[m][j] = fmaf(w, yb[j], a[m][j]);
          }
        }
        if (L >= 2) stash_prefetch(L - 2);
        float z[TMG][NCOL];
        stash_ld(L - 1, z);
        __syncthreads();   // the dW_L loop above reads cur, which the first reverse layer overwrites
#pragma unroll
        for (int m = 0; m < TMG; ++m) {
          float zz[NCOL];
#pragma unroll
          for (int pp = 0; pp < TPG; ++pp) act_bwd<C, DS, DIN, ACT>(&z[m][pp * C], &a[m][pp * C], &zz[pp * C]);
          row_store(zb, m, zz);
        }
      }
      for (int l = L - 1; l >= 1; --l) {
        if (l >= 2) stash_prefetch(l - 2);
        {   // A_{l-1} into ab
          float z[TMG][NCOL];
          stash_ld(l - 1, z);
          act_store(ab, z);
        }
        __syncthreads();
        // dW_l[i][k] += sum_pc Zb[i][pc] A_{l-1}[k][pc]: lanes take the input
        // neurons k = lane + 32 m, warp w the output neurons w + 8 r in blocks
        // of IB; even and odd columns summed in order apart (a fixed
        // summation order).  Per column pair a block loads IB broadcast and
        // TMG lane-strided 8-byte rows (IB + 2 TMG shared-memory wavefronts)
        // for IB TMG packed FMAs: with IB = 8 that stays under the SM's half a
        // wavefront per packed FMA; with 16-byte rows (4 columns per step) it
        // takes half the load instructions for the same sums.
        {
          float* const gw = g + sh.woff[l];
          const int nr = (W + 7) / 8;
          auto dw_block = [&](auto ibc, int r0) {
            constexpr int IB = decltype(ibc)::value;
            float2 acc[TMG][IB];   // .x the even, .y the odd columns
#pragma unroll
            for (int m = 0; m < TMG; ++m)
#pragma unroll
              for (int q = 0; q < IB; ++q) acc[m][q] = make_float2(0.f, 0.f);
            int irow[IB];
#pragma unroll
            for (int q = 0; q < IB; ++q) irow[q] = min(warp + 8 * (r0 + q), WP - 1) * RS;
            if constexpr (T::V4) {   // 4 columns per step: 16-byte rows (same per-column order)
              for (int pc = 0; pc < PC; pc += 4) {
                float4 zv[IB], av[TMG];
#pragma unroll
                for (int q = 0; q < IB; ++q) zv[q] = *reinterpret_cast<const float4*>(zb + irow[q] + pc);
#pragma unroll
                for (int m = 0; m < TMG; ++m) av[m] = *reinterpret_cast<const float4*>(ab + (lane + 32 * m) * RS + pc);
#pragma unroll
                for (int m = 0; m < TMG; ++m)
#pragma unroll
                  for (int q = 0; q < IB; ++q) {
                    acc[m][q] = __ffma2_rn(make_float2(zv[q].x, zv[q].y), make_float2(av[m].x, av[m].y), acc[m][q]);
                    acc[m][q] = __ffma2_rn(make_float2(zv[q].z, zv[q].w), make_float2(av[m].z, av[m].w), acc[m][q]);
                  }
              }
            } else {
              for (int pc = 0; pc < PC; pc += 2) {
                float2 zv[IB], av[TMG];
#pragma unroll
                for (int q = 0; q < IB; ++q) zv[q] = *reinterpret_cast<const float2*>(zb + irow[q] + pc);
#pragma unroll
                for (int m = 0; m < TMG; ++m) av[m] = *reinterpret_cast<const float2*>(ab + (lane + 32 * m) * RS + pc);
#pragma unroll
                for (int m = 0; m < TMG; ++m)
#pragma unroll
                  for (int q = 0; q < IB; ++q) acc[m][q] = __ffma2_rn(zv[q], av[m], acc[m][q]);
              }
            }
#pragma unroll
            for (int q = 0; q < IB; ++q) {
              const int i = warp + 8 * (r0 + q);
              if (i >= W) continue;
#pragma unroll
              for (int m = 0; m < TMG; ++m) {
                const int k = lane + 32 * m;
                if (k < W) grad_acc(gw + (size_t)i * W + k, acc[m][q].x + acc[m][q].y, first);
              }
            }
          };
          // row blocks that pad no row beyond the width: blocks of 5 for 16-byte
          // rows and a row count that 5 divides (25 at width 200), else
          // ceil(nr / 8) blocks of near-equal size, 5-8 rows at these widths
          // (measured against blocks of 8 and a tail of 4: -3 % at width 200,
          // -1.1 % at width 150)
          if (T::V4 && nr % 5 == 0) {
            for (int r0 = 0; r0 < nr; r0 += 5) dw_block(IntC<5>(), r0);
          } else {
            const int nb = (nr + 7) / 8;
            for (int bi = 0, r0 = 0; bi < nb; ++bi) {
              const int sz = nr / nb + (bi < nr % nb ? 1 : 0);
              switch (sz) {
                case 8: dw_block(IntC<8>(), r0); break;
                case 7: dw_block(IntC<7>(), r0); break;
                case 6: dw_block(IntC<6>(), r0); break;
                case 5: dw_block(IntC<5>(), r0); break;
                default:   // fewer than 5 rows per block: never at widths 129-224
                  for (int q = 0; q < sz; ++q) dw_block(IntC<1>(), r0 + q);
              }
              r0 += sz;
            }
          }
        }
        for (int e = t; e < W; e += NTW) {
          float s = 0.f;
          for (int p = 0; p < P; ++p) s += zb[e * RS + p * C];
          grad_acc(g + sh.boff[l] + e, s, first);
        }
        // A_{l-1} adjoint = W_l^T Zb_l (rows of W_l streamed: i, entries k);
        // the stash of layer l - 1 is loaded first, its latency under the
        // contraction
        float z[TMG][NCOL];
        stash_ld(l - 1, z);
        float a[TMG][NCOL];
        zero_acc(a);
        wide_contract<WP, C, NCOL, TV>(a, thT + (size_t)(l - 1) * 2 * W * WP + (size_t)W * WP, W, wch, zb, col0, ws);
        stash_discard(l);   // last read in the layer above, before this contraction's barriers
#pragma unroll
        for (int m = 0; m < TMG; ++m) {
          float zz[NCOL];
#pragma unroll
          for (int pp = 0; pp < TPG; ++pp) act_bwd<C, DS, DIN, ACT>(&z[m][pp * C], &a[m][pp * C], &zz[pp * C]);
          row_store(zb, m, zz);
        }
      }
      __syncthreads();
      stash_discard(0);
      // first affine map: dW_0[i][q] += sum_p (Zb_val xh_q + s_q Zb_q), db_0
      for (int e = t; e < W * DIN; e += NTW) {
        const int i = e / DIN, q = e % DIN;
        float s = 0.f;
        for (int p = 0; p < P; ++p) {
          s = fmaf(zb[i * RS + p * C], xh[p * 4 + q], s);
          if constexpr (JETS) s = fmaf(s_scale[q], zb[i * RS + p * C + 1 + q], s);
        }
        grad_acc(g + sh.woff[0] + e, s, first);
      }
      for (int e = t; e < W; e += NTW) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += zb[e * RS + p * C];
        grad_acc(g + sh.boff[0] + e, s, first);
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
  // after a time-out: the last copy issued into each buffer, waited for with
  // the same bound, before the block's shared memory is released
  if (t == 0 && s_wabort) {
    if (ws.issued0 > 0) mbar_wait_ok(&s_wbar[0], (ws.issued0 - 1) & 1);
    if (ws.issued1 > 0) mbar_wait_ok(&s_wbar[1], (ws.issued1 - 1) & 1);
  }
}

}  // namespace dk

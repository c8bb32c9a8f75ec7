// Tensor-core variant of the jet training kernel (width 128): the same work as
// k_pinn<128, DS, UNST, true, M_TRAIN, ACT> - per tile of 16 residual points,
// the forward jets through all layers, the Navier-Stokes residuals and L_PDE
// (Eqs. (5), (7)-(10)), and the reverse pass with the weight gradients of the
// item - with the three W x W contractions of every hidden layer on the
// tcgen05 tensor cores in compensated TF32 (3xTF32):
//
//   forward       Z_l       = W_l     a_{l-1}     M = 128 neurons, N = 16 C columns, K = 128
//   input adjoint abar_{l-1} = W_l^T  zbar_l      M = 128,         N = 16 C,         K = 128
//   weight grad   dW_l      = zbar_l  a_{l-1}^T   M = 128,         N = 128,          K = 16 C
//
// Every FP32 operand x is split into TF32 parts x = hi + lo (+ O(2^-22 |x|))
// and a product is accumulated as A_hi B_hi + (A_hi B_lo + A_lo B_hi) in FP32
// tensor-memory accumulators, which keeps the FP32-grade accuracy of the path
// (the A_lo B_lo term is below FP32 rounding).
//
// Layout.  512 threads; thread (warp w, lane) owns neuron 32 (w % 4) + lane -
// its lane of tensor memory - and the column quarter w / 4 (points
// 4 (w / 4) .. + 3 of the tile), so the jet recursion and its adjoint stay
// thread-local as in the FFMA kernel.  Columns are channel-major
// (n = c * 16 + p).  Tensor memory (512 columns): [0, 256) the A operand in
// hi / lo halves (W_l, or W_l^T, or zbar_l), [256, 384) and [384, 512) two
// accumulators: for the M x N products the main sum in the first and the
// corrections in the second, for the weight gradient the other way round.
// Shared memory: two operand regions in the 128-byte-swizzled K-major layout,
// [n][neuron] (a_{l-1} forward, zbar_l reverse; a warp's 32 neurons fill one
// 128-byte row, so the stores are conflict-free) and [neuron][n] (a_{l-1} for
// the weight gradient, one 16-byte chunk per store).  The next weight matrix
// is staged by a bulk copy into whichever region is idle while an MMA runs.
// The first affine map and the output layer (d_out rows) stay on FP32 FMA.
#pragma once
#include "pinn_kernels.cuh"
#include "tc.cuh"

namespace dk {

constexpr int NTC = 512;   // threads of the tensor-core kernels

template <int C>
struct TcTile {
  static constexpr int W = 128;
  static constexpr int P = 16;                        // points per tile
  static constexpr int NQ = NTC / 128;                // column groups (threads per neuron)
  static constexpr int HP = P / NQ;                   // points per thread
  static constexpr int NC = P * C;                    // columns, n = c * P + p
  static constexpr int KB = (NC + 31) / 32;           // 32-column blocks of [neuron][n]
  static constexpr uint32_t XT = (uint32_t)NC * 512;  // one [NC][128] tile (hi or lo), bytes
  static constexpr uint32_t ABT = (uint32_t)KB * 16384;   // one [128][NC] tile (hi or lo), bytes
  static constexpr uint32_t R1 = 2 * XT;              // [neuron][n] region
  static constexpr uint32_t SMALL = R1 + 2 * ABT;     // small tensors from here
  static constexpr int RSO = NC + 4;                  // row stride of a_{L-1} (FP32, in region R1)
  static_assert(HP == 4, "one float4 per channel and thread");
  static_assert(NC % 16 == 0 && NC <= 128, "accumulator columns");
  static_assert((size_t)W * RSO * 4 <= 2 * (size_t)ABT, "a_{L-1} buffer");
  static_assert((size_t)W * W * 4 <= 2 * (size_t)XT && (size_t)W * W * 4 <= 2 * (size_t)ABT, "weight staging");
};

template <int C, int DOUT>
constexpr size_t tc_smem_bytes(int L) {
  using T = TcTile<C>;
  return 1024 + T::SMALL +
         4 * ((size_t)2 * DOUT * T::NC + T::P * 4 + T::W * 4 + T::W + DOUT * T::W + 4 + T::NQ * T::W * 8 +
              (size_t)(L > 1 ? L - 1 : 0) * T::W);
}

// stash floats per CTA: per layer and thread C float4 (4 points x C channels)
template <int C>
constexpr long long tc_stash_floats(int L) { return (long long)L * C * NTC * 4; }

// A (tmem a_hi / a_lo) * B^T (smem b_hi / b_lo, K-major, 128-byte swizzle,
// 32-value K blocks blk bytes apart), K = 8 ksteps, 3xTF32: the main products
// A_hi B_hi accumulate in d, the correction products A_hi B_lo + A_lo B_hi in
// dx (the product is d + dx).  Each accumulator add of the tensor core rounds
// relative to the running sum; keeping the corrections (2^-11 smaller) apart
// leaves K / 8 such adds on the main sum instead of 3 K / 8.
__device__ __forceinline__ void mma3(uint32_t d, uint32_t dx, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                     uint32_t b_lo, uint32_t blk, int ksteps, uint32_t idesc) {
  for (int s = 0; s < ksteps; ++s) {
    const uint32_t bo = (uint32_t)(s >> 2) * blk + (uint32_t)(s & 3) * 32;
    const uint64_t bh = tc::desc_sw128(b_hi + bo), bl = tc::desc_sw128(b_lo + bo);
    const uint32_t acc = s > 0 ? 1u : 0u;
    tc::mma_ts(dx, a_hi + 8 * s, bl, idesc, acc);
    tc::mma_ts(dx, a_lo + 8 * s, bh, idesc, 1u);
    tc::mma_ts(d, a_hi + 8 * s, bh, idesc, acc);
  }
}

// Gradient accumulation into the item's slot: the first tile of an item
// stores, later tiles add with fire-and-forget reductions performed at L2 (no
// load round trip).  Every address has one owning thread, whose adds reach
// memory in program order, so the sums are deterministic.  (f32 reductions
// flush subnormal values, below 1.2e-38, to zero.)
__device__ __forceinline__ void gacc(float* p, float v, bool first) {
  if (first) *p = v;
  else asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
// A whole weight-gradient tile staged row-major in shared memory goes to the
// item's slot in one asynchronous bulk operation issued by one thread: a store
// for the item's first tile, an add performed at L2 for later ones.  The
// issuing thread waits for each operation to complete (its global writes
// included) before the staging region is reused, so the operations on an
// address are applied one at a time in tile order (deterministic sums).
// Both addresses are 16-byte aligned and `bytes` is a multiple of 16.
__device__ __forceinline__ void bulk_flush(float* gdst, uint32_t ssrc, uint32_t bytes, bool first) {
  if (first)
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc), "r"(bytes)
                 : "memory");
  else
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc),
                 "r"(bytes)
                 : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_flush_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// L2 residency of the per-CTA stash: a bulk prefetch of a contiguous block
// into L2 ahead of its loads, and a discard of its lines after their last
// read (the values are dead; a discarded line is never written back to DRAM).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void l2_discard(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Deterministic sum over the CTA of one float per thread (fixed order).
__device__ __forceinline__ float block_sum_tc(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NTC / 32; ++w) s += red[w];
  }
  return s;   // valid in thread 0
}

// MODE M_TRAIN: residual items (losses, reverse pass); MODE M_QUERY: jets of
// routed query points and their residuals (forward only, the anchored
// pressure of Eq. (18) by a second pass at x_anc for master nets).
template <int DS, int UNST, int ACT, int MODE = M_TRAIN>
__global__ void __launch_bounds__(NTC, 1)
    k_pinn_tc(const Shape sh, const Bufs b, const Item* __restrict__ items, const int* __restrict__ n_items_ptr) {
  constexpr int W = 128, DIN = DS + UNST, C = DIN + 2, DOUT = DS + 1;
  constexpr bool TRAIN = (MODE == M_TRAIN);
  using T = TcTile<C>;
  constexpr int P = T::P, HP = T::HP, NQ = T::NQ, NC = T::NC, RSO = T::RSO;
  constexpr int KQ = W / NQ;   // weight-row columns per thread
  constexpr uint32_t XT = T::XT, ABT = T::ABT;
  constexpr uint32_t IDN = tc::idesc_tf32(128, NC), IDW = tc::idesc_tf32(128, 128);
  constexpr uint32_t TLO = 128, TD = 256, TG = 384, TCOLS = 512;

  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t* const sb = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* const gX = sb;                 // [n][neuron] hi
  uint8_t* const gXl = sb + XT;           // [n][neuron] lo
  uint8_t* const gA = sb + T::R1;         // [neuron][n] hi
  uint8_t* const gAl = gA + ABT;          // [neuron][n] lo
  const uint32_t sX = tc::saddr(gX), sXl = tc::saddr(gXl), sA = tc::saddr(gA), sAl = tc::saddr(gAl);
  float* const outa = reinterpret_cast<float*>(gA);   // forward: a_{L-1} in FP32 [W][RSO]
  float* const ysm = reinterpret_cast<float*>(sb + T::SMALL);   // [DOUT][P * C] point-major
  float* const ybsm = ysm + DOUT * NC;
  float* const xh = ybsm + DOUT * NC;     // [P][4]
  float* const w0s = xh + P * 4;          // [W][4]
  float* const b0s = w0s + W * 4;         // [W]
  float* const wLs = b0s + W;             // [DOUT][W]
  float* const bLs = wLs + DOUT * W;      // [4]
  float* const xpart = bLs + 4;           // [NQ][W][8] column-group partial sums
  float* const bls = xpart + NQ * W * 8;  // [L-1][W]
  __shared__ __align__(8) uint64_t mbar;   // MMA completion
  __shared__ __align__(8) uint64_t dbar;   // drain after a time-out
  __shared__ __align__(8) uint64_t wbar;   // weight staging copies
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort;
  __shared__ float s_red[NTC / 32];
  __shared__ float s_scale[4];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int qd = warp & 3, hq = warp >> 2;
  const int nrn = qd * 32 + lane;                        // the thread's neuron = tensor-memory lane
  const int p0 = hq * HP;                                // the thread's first point
  const uint32_t lrow = (uint32_t)(qd * 32) << 16;       // lane field of the warp's accesses
  const int L = sh.L;
  const int n_items = *n_items_ptr;

  if (t == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&dbar, 1);
    mbar_init(&wbar, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::alloc(&s_tmem, TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  uint32_t phase = 0, wphase = 0;
  float4* const stash = reinterpret_cast<float4*>(b.stash + (TRAIN ? (size_t)blockIdx.x * b.stash_per_cta : 0));

  // MMA issue (one thread) and completion; after a time-out the remaining
  // MMAs and waits are skipped and the host sees ERR_TIMEOUT.
  auto issue = [&](uint32_t d, uint32_t dx, uint32_t bh, uint32_t bl, uint32_t blk, int ksteps, uint32_t idesc) {
    if (t == 0 && !s_abort) {
      mma3(d, dx, tm, tm + TLO, bh, bl, blk, ksteps, idesc);
      tc::commit(&mbar);
    }
  };
  auto wait_mma = [&]() {
    if (!*(volatile int*)&s_abort && !mbar_wait_ok(&mbar, phase & 1)) {
      s_abort = 1;
      atomicExch(b.err + ERR_TIMEOUT, 1);
    }
    ++phase;
    tc::fence_after();
  };
  // operands written by all threads -> visible to the MMA issued next
  auto publish = [&]() {
    tc::wait_st();
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  };
  // stash: one float4 per channel c (the thread's 4 points); layer l of the
  // CTA is one contiguous block of C * NTC float4
  constexpr uint32_t STASH_LAYER_BYTES = (uint32_t)C * NTC * 16;
  auto stash_prefetch = [&](int l) {
    if (t == 0) l2_prefetch(stash + (size_t)l * C * NTC, STASH_LAYER_BYTES);
  };
  auto stash_discard = [&](int l) {
    for (uint32_t o = (uint32_t)t * 128; o < STASH_LAYER_BYTES; o += NTC * 128)
      l2_discard(reinterpret_cast<const char*>(stash + (size_t)l * C * NTC) + o);
  };
  auto stash_st = [&](int l, const float (&h)[C][HP]) {
#pragma unroll
    for (int c = 0; c < C; ++c)
      stash[((size_t)l * C + c) * NTC + t] = make_float4(h[c][0], h[c][1], h[c][2], h[c][3]);
  };
  auto stash_ld = [&](int l, float (&h)[C][HP]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float4 v = stash[((size_t)l * C + c) * NTC + t];
      h[c][0] = v.x; h[c][1] = v.y; h[c][2] = v.z; h[c][3] = v.w;
    }
  };
  // activation jets of the thread's points from their stashed form
  auto act_pts = [&](const float (&h)[C][HP], float (&a)[C][HP]) {
#pragma unroll
    for (int u = 0; u < HP; ++u) {
      float hz[C], av[C];
#pragma unroll
      for (int c = 0; c < C; ++c) hz[c] = h[c][u];
      act_from_stash<C, DS, DIN, ACT>(hz, av);
#pragma unroll
      for (int c = 0; c < C; ++c) a[c][u] = av[c];
    }
  };
  // value of the thread's point u, channel c, neuron nrn -> [n][neuron]
  // operand (hi, lo): row n = c P + p0 + u, column nrn
  auto put_row = [&](int c, int u, float v) {
    const int n = c * P + p0 + u;
    const uint32_t off = (uint32_t)qd * (NC * 128) + (uint32_t)(n >> 3) * 1024 + (uint32_t)(n & 7) * 128 +
                         ((uint32_t)((lane >> 2) ^ (n & 7)) << 4) + (uint32_t)(lane & 3) * 4;
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    *reinterpret_cast<float*>(gX + off) = hi;
    *reinterpret_cast<float*>(gXl + off) = lo;
  };
  // the thread's 4 points of channel c -> [neuron][n] operand (hi, lo): row
  // nrn, columns n = c P + p0 .. + 3 (one 16-byte chunk)
  auto put_col4 = [&](int c, const float (&v)[HP]) {
    const int chunk = (c & 1) * 4 + hq;
    const uint32_t off = (uint32_t)(c >> 1) * 16384 + (uint32_t)(nrn >> 3) * 1024 + (uint32_t)(nrn & 7) * 128 +
                         ((uint32_t)(chunk ^ (nrn & 7)) << 4);
    float4 h4, l4;
    tc::split_tf32(v[0], h4.x, l4.x);
    tc::split_tf32(v[1], h4.y, l4.y);
    tc::split_tf32(v[2], h4.z, l4.z);
    tc::split_tf32(v[3], h4.w, l4.w);
    *reinterpret_cast<float4*>(gA + off) = h4;
    *reinterpret_cast<float4*>(gAl + off) = l4;
  };
  // KQ columns (the thread's quarter) of row nrn of a W x W matrix -> tensor
  // memory hi / lo, from global memory ...
  auto put_w = [&](const float* row) {
    float hi[KQ], lo[KQ];
#pragma unroll
    for (int j = 0; j < KQ; j += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(row + j));
      tc::split_tf32(v.x, hi[j], lo[j]);
      tc::split_tf32(v.y, hi[j + 1], lo[j + 1]);
      tc::split_tf32(v.z, hi[j + 2], lo[j + 2]);
      tc::split_tf32(v.w, hi[j + 3], lo[j + 3]);
    }
    tc::st32(tm + lrow + (uint32_t)(hq * KQ), hi);
    tc::st32(tm + lrow + TLO + (uint32_t)(hq * KQ), lo);
  };
  // ... or from a copy staged in shared memory whose element (row nrn,
  // column k) sits at ws[k W + nrn] (a transposed copy): a warp reads 128
  // consecutive bytes per column
  auto put_w_staged = [&](const float* ws) {
    mbar_wait(&wbar, wphase & 1, b.err);
    ++wphase;
    float hi[KQ], lo[KQ];
#pragma unroll
    for (int j = 0; j < KQ; ++j) tc::split_tf32(ws[(hq * KQ + j) * W + nrn], hi[j], lo[j]);
    tc::st32(tm + lrow + (uint32_t)(hq * KQ), hi);
    tc::st32(tm + lrow + TLO + (uint32_t)(hq * KQ), lo);
  };
  // activations -> next forward operand, or a_{L-1} in FP32
  auto put_act = [&](int l, const float (&a)[C][HP]) {
    if (l + 1 < L) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int u = 0; u < HP; ++u) put_row(c, u, a[c][u]);
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c)
        *reinterpret_cast<float4*>(outa + nrn * RSO + c * P + p0) = make_float4(a[c][0], a[c][1], a[c][2], a[c][3]);
    }
  };
  // M x N result (main + corrections) of the thread's points
  auto ld_result = [&](float (&r)[C][HP]) {
    float v[C][4], x[C][4];   // channel c: columns c P + p0 .. + 3 of each accumulator
    tc::ld4_rows<C>(tm + lrow + TD + (uint32_t)p0, (uint32_t)P, v);
    tc::ld4_rows<C>(tm + lrow + TG + (uint32_t)p0, (uint32_t)P, x);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int u = 0; u < HP; ++u) r[c][u] = v[c][u] + x[c][u];
  };

  for (;;) {
    if (t == 0) s_item = atomicAdd(b.counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items || s_abort) break;
    const Item item = items[it];
    const int net = item.net;
    const float* const th = b.theta + (size_t)net * sh.npp;
    const float* const thT = b.thetaT + (size_t)net * sh.nTp;
    const NetInfo ni = b.nets[net];
    for (int e = t; e < W * DIN; e += NTC) w0s[(e / DIN) * 4 + e % DIN] = th[sh.woff[0] + e];
    for (int e = t; e < W; e += NTC) b0s[e] = th[sh.boff[0] + e];
    for (int e = t; e < (L - 1) * W; e += NTC) bls[e] = th[sh.boff[1 + e / W] + e % W];
    for (int e = t; e < DOUT * W; e += NTC) wLs[e] = th[sh.woff[L] + e];
    if (t < DOUT) bLs[t] = th[sh.boff[L] + t];
    // scale from global memory: a run-time index into the local copy ni would
    // move that copy to the stack
    if (t < 4) s_scale[t] = t < DIN ? b.nets[net].scale[t] : 0.f;
    double lsum0 = 0.0;   // thread 0: sum of r^2 over the item
    const int npass = (!TRAIN && ni.master && !b.q_jets) ? 2 : 1;

    for (int sub = 0; sub < item.count; sub += P) {
      const int npts = min(P, item.count - sub);
      const bool first = (sub == 0);
      float pkeep = 0.f;   // query: raw pressure of a master point (thread t = point)
     for (int pass = 0; pass < npass; ++pass) {
      // ---- inputs mapped to the net's box: xh = (x - c) * s
      if (t < P) {
        const bool valid = t < npts;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
          const float* src = TRAIN ? b.res_pts + (size_t)(item.begin + sub + t) * DIN
                                   : b.q_pts + (size_t)b.q_perm[item.begin + sub + t] * DIN;
#pragma unroll
          for (int q = 0; q < DIN; ++q) x[q] = src[q];
          if (pass == 1) {   // p(x_anc, t) at the point's time
#pragma unroll
            for (int q = 0; q < DS; ++q) x[q] = sh.anchor[q];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) xh[t * 4 + q] = (valid && q < DIN) ? (x[q] - ni.center[q]) * ni.scale[q] : 0.f;
      }
      __syncthreads();
      // ---- first affine map (FP32): z = W0 xh + b0, d_q z = s_q W0[:, q], lap z = 0
      {
        float w[DIN];
#pragma unroll
        for (int q = 0; q < DIN; ++q) w[q] = w0s[nrn * 4 + q];
        const float bias = b0s[nrn];
        float h[C][HP], a[C][HP];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          const int p = p0 + u;
          float v = bias;
#pragma unroll
          for (int q = 0; q < DIN; ++q) v = fmaf(w[q], xh[p * 4 + q], v);
          h[0][u] = stash_value<ACT>(v);
#pragma unroll
          for (int q = 0; q < DIN; ++q) h[1 + q][u] = w[q] * s_scale[q];
          h[C - 1][u] = 0.f;
        }
        if (TRAIN) stash_st(0, h);
        act_pts(h, a);
        put_act(0, a);
      }
      // ---- hidden layers on the tensor cores (W_l rows: lane = output neuron)
      if (L > 1) put_w(th + sh.woff[1] + (size_t)nrn * W + hq * KQ);
      for (int l = 1; l < L; ++l) {
        publish();
        issue(tm + TD, tm + TG, sX, sXl, NC * 128, W / 8, IDN);
        // W_{l+1}^T is staged into the (idle) weight-gradient operand region
        // while the MMA runs, and moved to tensor memory once it has completed
        if (t == 0 && l + 1 < L) bulk_load(gA, thT + (size_t)l * W * W, W * W * 4, &wbar);
        wait_mma();
        float h[C][HP], a[C][HP];
        ld_result(h);
        if (l + 1 < L) put_w_staged(reinterpret_cast<const float*>(gA));
        const float bias = bls[(l - 1) * W + nrn];
#pragma unroll
        for (int u = 0; u < HP; ++u) h[0][u] = stash_value<ACT>(h[0][u] + bias);
        if (TRAIN) stash_st(l, h);
        act_pts(h, a);
        put_act(l, a);
      }
      __syncthreads();
      // ---- output layer (FP32): Y[j][p][c] = W_L[j] . a_{L-1}[.][p][c] (+ b_L on values)
      {
        constexpr int PAIRS = DOUT * P;
        constexpr int KS = NTC / PAIRS >= 8 ? 8 : (NTC / PAIRS >= 4 ? 4 : 2);
        for (int pr = t / KS; pr < PAIRS; pr += NTC / KS) {
          const int j = pr / P, p = pr % P, lk = t % KS;
          float acc[C];
#pragma unroll
          for (int c = 0; c < C; ++c) acc[c] = 0.f;
          for (int k = lk; k < W; k += KS) {
            const float w = wLs[j * W + k];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fmaf(w, outa[k * RSO + c * P + p], acc[c]);
          }
#pragma unroll
          for (int o = KS / 2; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
          if (lk == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) ysm[j * NC + p * C + c] = acc[c] + (c == 0 ? bLs[j] : 0.f);
          }
        }
      }
      __syncthreads();
      if constexpr (!TRAIN) {   // query outputs: (u, p) and the residuals
        if (t < P && t < npts) {
          float Y[DOUT][C];
#pragma unroll
          for (int j = 0; j < DOUT; ++j)
#pragma unroll
            for (int c = 0; c < C; ++c) Y[j][c] = ysm[j * NC + t * C + c];
          float* o = b.q_out + (size_t)b.q_perm[item.begin + sub + t] * b.q_w;
          if (b.q_jets) {   // the net's own output jets, row [j][c] (one pass)
#pragma unroll
            for (int j = 0; j < DOUT; ++j)
#pragma unroll
              for (int c = 0; c < C; ++c) o[j * C + c] = Y[j][c];
          } else if (pass == 0) {
#pragma unroll
            for (int j = 0; j < DS; ++j) o[j] = Y[j][0];
            if (npass == 1) o[DS] = Y[DS][0] + sh.p_ref;
            else pkeep = Y[DS][0];
            float r[DS + 1];
            ns_residual<DS, UNST, C>(Y, sh.nu, r);
#pragma unroll
            for (int j = 0; j <= DS; ++j) o[DOUT + j] = r[j];
          } else {
            o[DS] = (pkeep - Y[DS][0]) + sh.p_ref;
          }
        }
        __syncthreads();
        continue;
      }
      // ---- residuals, L_PDE and the output adjoint seeds (thread = point)
      float l0 = 0.f;
      if (t < P) {
        const bool valid = t < npts;
        float Y[DOUT][C], Yb[DOUT][C];
#pragma unroll
        for (int j = 0; j < DOUT; ++j)
#pragma unroll
          for (int c = 0; c < C; ++c) {
            Y[j][c] = ysm[j * NC + t * C + c];
            Yb[j][c] = 0.f;
          }
        const float r2 = pde_seed<DS, UNST, C>(Y, sh.nu, valid ? 2.f * sh.lam_pde * ni.inv_npde : 0.f, Yb);
        l0 = valid ? r2 : 0.f;
#pragma unroll
        for (int j = 0; j < DOUT; ++j)
#pragma unroll
          for (int c = 0; c < C; ++c) ybsm[j * NC + t * C + c] = Yb[j][c];
      }
      {
        const float s = block_sum_tc(l0, s_red);
        if (t == 0) lsum0 += (double)s;
      }
      __syncthreads();
     }   // pass
      if constexpr (!TRAIN) continue;
      if (b.no_reverse) continue;

      // ================= reverse pass =================
      float* const g = b.grad_part + (size_t)item.slot * sh.npp;
      // the stashed form of layer l is loaded one layer ahead (hsn)
      float hsn[C][HP];
      if (L > 1) stash_prefetch(L - 2);
      stash_ld(L - 1, hsn);
      // W_{L-1}^T rows (lane = input neuron)
      if (L > 1) put_w(thT + (size_t)(L - 2) * W * W + (size_t)nrn * W + hq * KQ);
      // output layer: dW_L[j][k] = sum_{p,c} Yb[j][p][c] a_{L-1}[k][p][c], db_L
      for (int e = t; e < DOUT * W; e += NTC) {
        const int j = e / W, k = e % W;
        float s = 0.f;
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int c = 0; c < C; ++c) s = fmaf(ybsm[j * NC + p * C + c], outa[k * RSO + c * P + p], s);
        gacc(g + sh.woff[L] + e, s, first);
      }
      if (t < DOUT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += ybsm[t * NC + p * C];
        gacc(g + sh.boff[L] + t, s, first);
      }
      // adjoint of a_{L-1} for the thread's neuron and points: W_L^T Yb
      float ab[C][HP];
      {
        float wl[DOUT];
#pragma unroll
        for (int j = 0; j < DOUT; ++j) wl[j] = wLs[j * W + nrn];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          const int p = p0 + u;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < DOUT; ++j) v = fmaf(wl[j], ybsm[j * NC + p * C + c], v);
            ab[c][u] = v;
          }
        }
      }
      for (int l = L - 1; l >= 1; --l) {
        // zbar_l = adjoint of the activation at layer l
        float zb[C][HP];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float hz[C], av[C], zz[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            hz[c] = hsn[c][u];
            av[c] = ab[c][u];
          }
          act_bwd<C, DS, DIN, ACT>(hz, av, zz);
#pragma unroll
          for (int c = 0; c < C; ++c) zb[c][u] = zz[c];
        }
        xpart[(hq * W + nrn) * 8] = (zb[0][0] + zb[0][1]) + (zb[0][2] + zb[0][3]);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int u = 0; u < HP; ++u) put_row(c, u, zb[c][u]);   // zbar_l as [n][out]
        if (t == 0) bulk_flush_wait();   // the previous layer's tile has left the staging region
        publish();
        issue(tm + TD, tm + TG, sX, sXl, NC * 128, W / 8, IDN);   // abar_{l-1} = W_l^T zbar_l
        stash_discard(l);   // its last reads (hsn) precede the barrier above
        if (l > 1) stash_prefetch(l - 2);
        // meanwhile: a_{l-1} as the [in][n] operand of the weight gradient, and db_l
        stash_ld(l - 1, hsn);
        {
          float a[C][HP];
          act_pts(hsn, a);
#pragma unroll
          for (int c = 0; c < C; ++c) put_col4(c, a[c]);
        }
        if (hq == 0) {
          float s = 0.f;
#pragma unroll
          for (int q = 0; q < NQ; ++q) s += xpart[(q * W + nrn) * 8];
          gacc(g + sh.boff[l] + nrn, s, first);
        }
        wait_mma();
        // W_{l-1} is staged into the [n][neuron] region (idle until the next
        // layer) while the weight-gradient MMA runs
        if (t == 0 && l > 1) bulk_load(gX, th + sh.woff[l - 1], W * W * 4, &wbar);
        // zbar_l -> tensor memory (A operand of the weight gradient, lane = output neuron)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float hv[4], lv[4];
#pragma unroll
          for (int u = 0; u < HP; ++u) tc::split_tf32(zb[c][u], hv[u], lv[u]);
          tc::st4(tm + lrow + (uint32_t)(c * P + p0), hv);
          tc::st4(tm + lrow + TLO + (uint32_t)(c * P + p0), lv);
        }
        ld_result(ab);
        publish();
        issue(tm + TG, tm + TD, sA, sAl, 16384, NC / 8, IDW);    // dW_l = zbar_l a_{l-1}^T
        wait_mma();
        {
          // the thread's 32 columns of row nrn as 8 float4 chunks, then an
          // 8 x 8 transpose of chunks among each group of 8 lanes, so that the
          // 8 lanes of a group write one 128-byte row segment per instruction
          // (full sectors) instead of 8 rows 16 bytes each
          static_assert(KQ == 32, "8 chunks per thread");
          float4 q[8];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            float v[16], x[16];
            tc::ld16_pair(tm + lrow + TG + (uint32_t)(hq * KQ + h2 * 16), tm + lrow + TD + (uint32_t)(hq * KQ + h2 * 16),
                          v, x);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              q[h2 * 4 + j] = make_float4(v[4 * j] + x[4 * j], v[4 * j + 1] + x[4 * j + 1], v[4 * j + 2] + x[4 * j + 2],
                                          v[4 * j + 3] + x[4 * j + 3]);
          }
#pragma unroll
          for (int sx = 4; sx >= 1; sx >>= 1) {
            const bool up = (lane & sx) != 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              if ((c & sx) == 0) {
                const float4 snd = up ? q[c] : q[c | sx];
                float4 rcv;
                rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, sx);
                rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, sx);
                rcv.z = __shfl_xor_sync(0xffffffffu, snd.z, sx);
                rcv.w = __shfl_xor_sync(0xffffffffu, snd.w, sx);
                if (up) q[c] = rcv;
                else q[c | sx] = rcv;
              }
            }
          }
          // lane (8 gr + j) now holds chunk j of the rows of lanes 8 gr + c:
          // the 8 lanes of a group store one 128-byte row segment (one
          // wavefront) of the row-major tile, staged in the [neuron][n]
          // operand region (idle until the next layer's activation operand)
          const int row0 = qd * 32 + (lane & ~7);
          float* const sw = reinterpret_cast<float*>(gA) + row0 * W + hq * KQ + 4 * (lane & 7);
#pragma unroll
          for (int c = 0; c < 8; ++c) *reinterpret_cast<float4*>(sw + c * W) = q[c];
          tc::fence_smem_async();
        }
        // the weight-gradient MMA (A operand zbar_l) has completed
        if (l > 1) put_w_staged(reinterpret_cast<const float*>(gX));
        __syncthreads();   // the staged tile is whole; reads of the staged weights precede the next zbar rows
        if (t == 0) bulk_flush(g + sh.woff[l], sA, W * W * 4, first);
      }
      // first affine map: dW_0[i][q] += sum_p (zbar_val xh_q + s_q zbar_q), db_0
      __syncthreads();
      stash_discard(0);
      {
        float part[DIN + 1];
#pragma unroll
        for (int q = 0; q <= DIN; ++q) part[q] = 0.f;
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float hz[C], av[C], zz[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            hz[c] = hsn[c][u];
            av[c] = ab[c][u];
          }
          act_bwd<C, DS, DIN, ACT>(hz, av, zz);
          const int p = p0 + u;
#pragma unroll
          for (int q = 0; q < DIN; ++q) {
            part[q] = fmaf(zz[0], xh[p * 4 + q], part[q]);
            part[q] = fmaf(s_scale[q], zz[1 + q], part[q]);
          }
          part[DIN] += zz[0];
        }
#pragma unroll
        for (int q = 0; q <= DIN; ++q) xpart[(hq * W + nrn) * 8 + q] = part[q];
      }
      if (t == 0) bulk_flush_wait();   // layer 1's tile has left the staging region
      __syncthreads();
      if (hq == 0) {
#pragma unroll
        for (int q = 0; q <= DIN; ++q) {
          float s = 0.f;
#pragma unroll
          for (int r = 0; r < NQ; ++r) s += xpart[(r * W + nrn) * 8 + q];
          gacc(q < DIN ? g + sh.woff[0] + nrn * DIN + q : g + sh.boff[0] + nrn, s, first);
        }
      }
      __syncthreads();
    }   // sub-tiles
    if (TRAIN && t == 0) {
      double* lp = b.loss_part + (size_t)item.slot * LP;
      for (int q = 0; q < LP; ++q) lp[q] = 0.0;
      lp[1] = lsum0;
    }
  }   // items
  // drain: after a time-out, give the outstanding MMAs a bounded time before
  // the tensor memory is released.  The waits skipped after the time-out leave
  // mbar's parity unknown, so the drain commits to a barrier of its own (a
  // commit tracks every MMA the thread issued before it).
  if (t == 0 && s_abort) {
    tc::commit(&dbar);
    mbar_wait_ok(&dbar, 0);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::dealloc(tm, TCOLS);
}

}  // namespace dk

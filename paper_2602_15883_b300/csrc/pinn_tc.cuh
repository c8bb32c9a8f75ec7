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
// and a product is accumulated as A_hi B_lo + A_lo B_hi + A_hi B_hi in the
// FP32 tensor-memory accumulator, which keeps the FP32-grade accuracy of the
// path (the A_lo B_lo term is below FP32 rounding).
//
// Layout.  Thread (warp w, lane) owns neuron 32 (w % 4) + lane - its lane of
// tensor memory - and the column half w / 4 (points 8 (w / 4) .. + 7 of the
// tile), so the jet recursion and its adjoint stay thread-local as in the FFMA
// kernel.  Columns are channel-major (n = c * 16 + p).  Tensor memory (512
// columns): [0, 256) the A operand in hi / lo halves (W_l, or W_l^T, or
// zbar_l), [256, 384) and [384, 512) two accumulators: for the M x N
// products the main sum in the first and the 3xTF32 corrections in the
// second, for the weight gradient the other way round.  Shared memory: two operand regions in the 128-byte-swizzled
// K-major layout, [n][neuron] (a_{l-1} forward, zbar_l reverse; a warp's 32
// neurons fill one 128-byte row, so the stores are conflict-free) and
// [neuron][n] (a_{l-1} for the weight gradient, one 16-byte chunk per store).
// The first affine map and the output layer (d_out rows) stay on FP32 FMA.
#pragma once
#include "pinn_kernels.cuh"
#include "tc.cuh"

namespace dk {

template <int C>
struct TcTile {
  static constexpr int W = 128;
  static constexpr int P = 16;                        // points per tile
  static constexpr int HP = 8;                        // points per column half
  static constexpr int NC = P * C;                    // columns, n = c * P + p
  static constexpr int KB = (NC + 31) / 32;           // 32-column blocks of [neuron][n]
  static constexpr uint32_t XT = (uint32_t)NC * 512;  // one [NC][128] tile (hi or lo), bytes
  static constexpr uint32_t ABT = (uint32_t)KB * 16384;   // one [128][NC] tile (hi or lo), bytes
  static constexpr uint32_t R1 = 2 * XT;              // [neuron][n] region
  static constexpr uint32_t SMALL = R1 + 2 * ABT;     // small tensors from here
  static constexpr int RSO = NC + 4;                  // row stride of a_{L-1} (FP32, in region R1)
  static constexpr int SQ = 2 * C;                    // stashed float4 per thread per layer
  static_assert(NC % 16 == 0 && NC <= 128, "accumulator columns");
  static_assert((size_t)W * RSO * 4 <= 2 * (size_t)ABT, "a_{L-1} buffer");
};

template <int C, int DOUT>
constexpr size_t tc_smem_bytes(int L) {
  using T = TcTile<C>;
  return 1024 + T::SMALL +
         4 * ((size_t)2 * DOUT * T::NC + T::P * 4 + T::W * 4 + T::W + DOUT * T::W + 4 + 2 * T::W * 8 +
              (size_t)(L > 1 ? L - 1 : 0) * T::W);
}

// stash floats per CTA
template <int C>
constexpr long long tc_stash_floats(int L) { return (long long)L * TcTile<C>::SQ * NT * 4; }

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

template <int DS, int UNST, int ACT>
__global__ void __launch_bounds__(NT, 1)
    k_pinn_tc(const Shape sh, const Bufs b, const Item* __restrict__ items, const int* __restrict__ n_items_ptr) {
  constexpr int W = 128, DIN = DS + UNST, C = DIN + 2, DOUT = DS + 1;
  using T = TcTile<C>;
  constexpr int P = T::P, HP = T::HP, NC = T::NC, RSO = T::RSO, SQ = T::SQ;
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
  float* const xpart = bLs + 4;           // [2][W][8] column-half partial sums
  float* const bls = xpart + 2 * W * 8;   // [L-1][W]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort;
  __shared__ float s_red[NT / 32];
  __shared__ float s_scale[4];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int qd = warp & 3, hf = warp >> 2;
  const int nrn = qd * 32 + lane;                        // the thread's neuron = tensor-memory lane
  const uint32_t lrow = (uint32_t)(qd * 32) << 16;       // lane field of the warp's accesses
  const int L = sh.L;
  const int n_items = *n_items_ptr;

  if (t == 0) {
    mbar_init(&mbar, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::alloc(&s_tmem, TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  uint32_t phase = 0;
  float4* const stash = reinterpret_cast<float4*>(b.stash + (size_t)blockIdx.x * b.stash_per_cta);

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
  // stash: float4 q = (channel c, points 4 j .. 4 j + 3 of the thread's half), q = 2 c + j
  auto stash_st4 = [&](int l, int j, const float (&h)[C][4]) {
#pragma unroll
    for (int c = 0; c < C; ++c)
      stash[((size_t)l * SQ + 2 * c + j) * NT + t] = make_float4(h[c][0], h[c][1], h[c][2], h[c][3]);
  };
  auto stash_ld4 = [&](int l, int j, float (&h)[C][4]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float4 v = stash[((size_t)l * SQ + 2 * c + j) * NT + t];
      h[c][0] = v.x; h[c][1] = v.y; h[c][2] = v.z; h[c][3] = v.w;
    }
  };
  // activation jets of 4 points from their stashed form
  auto act4 = [&](const float (&h)[C][4], float (&a)[C][4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float hz[C], av[C];
#pragma unroll
      for (int c = 0; c < C; ++c) hz[c] = h[c][u];
      act_from_stash<C, DS, DIN, ACT>(hz, av);
#pragma unroll
      for (int c = 0; c < C; ++c) a[c][u] = av[c];
    }
  };
  // value of point pp (of the thread's half), channel c, neuron nrn -> [n][neuron]
  // operand (hi, lo): row n = c P + 8 hf + pp (n % 8 = pp), column nrn
  auto put_row = [&](int c, int pp, float v) {
    const int n = c * P + hf * HP + pp;
    const uint32_t off = (uint32_t)qd * (NC * 128) + (uint32_t)(n >> 3) * 1024 + (uint32_t)pp * 128 +
                         ((uint32_t)((lane >> 2) ^ pp) << 4) + (uint32_t)(lane & 3) * 4;
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    *reinterpret_cast<float*>(gX + off) = hi;
    *reinterpret_cast<float*>(gXl + off) = lo;
  };
  // 4 points (group j) of channel c -> [neuron][n] operand (hi, lo): row nrn,
  // columns n = c P + 8 hf + 4 j .. + 3 (one 16-byte chunk)
  auto put_col4 = [&](int c, int j, const float (&v)[4]) {
    const int chunk = (c & 1) * 4 + hf * 2 + j;
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
  // 64 columns (the thread's half) of row nrn of a W x W matrix -> tensor memory hi / lo
  auto put_w = [&](const float* row) {
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(row + h2 * 32 + j));
        tc::split_tf32(v.x, hi[j], lo[j]);
        tc::split_tf32(v.y, hi[j + 1], lo[j + 1]);
        tc::split_tf32(v.z, hi[j + 2], lo[j + 2]);
        tc::split_tf32(v.w, hi[j + 3], lo[j + 3]);
      }
      tc::st32(tm + lrow + (uint32_t)(hf * 64 + h2 * 32), hi);
      tc::st32(tm + lrow + TLO + (uint32_t)(hf * 64 + h2 * 32), lo);
    }
  };
  // activations of 4 points (group j) -> next forward operand, or a_{L-1} in FP32
  auto put_act4 = [&](int l, int j, const float (&a)[C][4]) {
    if (l + 1 < L) {
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u) put_row(c, 4 * j + u, a[c][u]);
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c)
        *reinterpret_cast<float4*>(outa + nrn * RSO + c * P + hf * HP + 4 * j) =
            make_float4(a[c][0], a[c][1], a[c][2], a[c][3]);
    }
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
    for (int e = t; e < W * DIN; e += NT) w0s[(e / DIN) * 4 + e % DIN] = th[sh.woff[0] + e];
    for (int e = t; e < W; e += NT) b0s[e] = th[sh.boff[0] + e];
    for (int e = t; e < (L - 1) * W; e += NT) bls[e] = th[sh.boff[1 + e / W] + e % W];
    for (int e = t; e < DOUT * W; e += NT) wLs[e] = th[sh.woff[L] + e];
    if (t < DOUT) bLs[t] = th[sh.boff[L] + t];
    if (t < 4) s_scale[t] = t < DIN ? ni.scale[t] : 0.f;
    double lsum0 = 0.0;   // thread 0: sum of r^2 over the item

    for (int sub = 0; sub < item.count; sub += P) {
      const int npts = min(P, item.count - sub);
      const bool first = (sub == 0);
      // ---- inputs mapped to the net's box: xh = (x - c) * s
      if (t < P) {
        const bool valid = t < npts;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
          const float* src = b.res_pts + (size_t)(item.begin + sub + t) * DIN;
#pragma unroll
          for (int q = 0; q < DIN; ++q) x[q] = src[q];
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
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float h[C][4], a[C][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int p = hf * HP + 4 * j + u;
            float v = bias;
#pragma unroll
            for (int q = 0; q < DIN; ++q) v = fmaf(w[q], xh[p * 4 + q], v);
            h[0][u] = stash_value<ACT>(v);
#pragma unroll
            for (int q = 0; q < DIN; ++q) h[1 + q][u] = w[q] * s_scale[q];
            h[C - 1][u] = 0.f;
          }
          stash_st4(0, j, h);
          act4(h, a);
          put_act4(0, j, a);
        }
      }
      // ---- hidden layers on the tensor cores
      for (int l = 1; l < L; ++l) {
        put_w(th + sh.woff[l] + (size_t)nrn * W + hf * 64);   // lane = output neuron
        publish();
        issue(tm + TD, tm + TG, sX, sXl, NC * 128, W / 8, IDN);
        wait_mma();
        const float bias = bls[(l - 1) * W + nrn];
        float d8[C][8];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float x8[8];
          tc::ld8(tm + lrow + TD + (uint32_t)(c * P + hf * HP), d8[c]);
          tc::ld8(tm + lrow + TG + (uint32_t)(c * P + hf * HP), x8);
#pragma unroll
          for (int u = 0; u < 8; ++u) d8[c][u] += x8[u];
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float h[C][4], a[C][4];
#pragma unroll
          for (int c = 0; c < C; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) h[c][u] = d8[c][4 * j + u];
#pragma unroll
          for (int u = 0; u < 4; ++u) h[0][u] = stash_value<ACT>(h[0][u] + bias);
          stash_st4(l, j, h);
          act4(h, a);
          put_act4(l, j, a);
        }
      }
      __syncthreads();
      // ---- output layer (FP32): Y[j][p][c] = W_L[j] . a_{L-1}[.][p][c] (+ b_L on values)
      {
        constexpr int PAIRS = DOUT * P;
        constexpr int KS = NT / PAIRS >= 4 ? 4 : (NT / PAIRS >= 2 ? 2 : 1);
        for (int pr = t / KS; pr < PAIRS; pr += NT / KS) {
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
        const float s = block_sum(l0, s_red);
        if (t == 0) lsum0 += (double)s;
      }
      __syncthreads();
      if (b.no_reverse) continue;

      // ================= reverse pass =================
      float* const g = b.grad_part + (size_t)item.slot * sh.npp;
      // output layer: dW_L[j][k] = sum_{p,c} Yb[j][p][c] a_{L-1}[k][p][c], db_L
      for (int e = t; e < DOUT * W; e += NT) {
        const int j = e / W, k = e % W;
        float s = 0.f;
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int c = 0; c < C; ++c) s = fmaf(ybsm[j * NC + p * C + c], outa[k * RSO + c * P + p], s);
        grad_rmw(g + sh.woff[L] + e, s, first);
      }
      if (t < DOUT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += ybsm[t * NC + p * C];
        grad_rmw(g + sh.boff[L] + t, s, first);
      }
      // adjoint of a_{L-1} for the thread's neuron and points: W_L^T Yb
      float ab[C][HP];
      {
        float wl[DOUT];
#pragma unroll
        for (int j = 0; j < DOUT; ++j) wl[j] = wLs[j * W + nrn];
#pragma unroll
        for (int pp = 0; pp < HP; ++pp) {
          const int p = hf * HP + pp;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < DOUT; ++j) v = fmaf(wl[j], ybsm[j * NC + p * C + c], v);
            ab[c][pp] = v;
          }
        }
      }
      for (int l = L - 1; l >= 1; --l) {
        // zbar_l = adjoint of the activation at layer l (stashed jets)
        float zb[C][HP];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float hs[C][4];
          stash_ld4(l, j, hs);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float hz[C], av[C], zz[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              hz[c] = hs[c][u];
              av[c] = ab[c][4 * j + u];
            }
            act_bwd<C, DS, DIN, ACT>(hz, av, zz);
#pragma unroll
            for (int c = 0; c < C; ++c) zb[c][4 * j + u] = zz[c];
          }
        }
        {
          float s = 0.f;
#pragma unroll
          for (int pp = 0; pp < HP; ++pp) s += zb[0][pp];
          xpart[(hf * W + nrn) * 8] = s;
        }
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int pp = 0; pp < HP; ++pp) put_row(c, pp, zb[c][pp]);   // zbar_l as [n][out]
        put_w(thT + (size_t)(l - 1) * W * W + (size_t)nrn * W + hf * 64);   // W_l^T: lane = input neuron
        publish();
        issue(tm + TD, tm + TG, sX, sXl, NC * 128, W / 8, IDN);   // abar_{l-1} = W_l^T zbar_l
        // meanwhile: a_{l-1} as the [in][n] operand of the weight gradient, and db_l
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float hs[C][4], a[C][4];
          stash_ld4(l - 1, j, hs);
          act4(hs, a);
#pragma unroll
          for (int c = 0; c < C; ++c) put_col4(c, j, a[c]);
        }
        if (hf == 0) grad_rmw(g + sh.boff[l] + nrn, xpart[nrn * 8] + xpart[(W + nrn) * 8], first);
        wait_mma();
        // zbar_l -> tensor memory (A operand of the weight gradient, lane = output neuron)
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float hv[8], lv[8];
#pragma unroll
          for (int pp = 0; pp < HP; ++pp) tc::split_tf32(zb[c][pp], hv[pp], lv[pp]);
          tc::st8(tm + lrow + (uint32_t)(c * P + hf * HP), hv);
          tc::st8(tm + lrow + TLO + (uint32_t)(c * P + hf * HP), lv);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          float v[8], x8[8];
          tc::ld8(tm + lrow + TD + (uint32_t)(c * P + hf * HP), v);
          tc::ld8(tm + lrow + TG + (uint32_t)(c * P + hf * HP), x8);
#pragma unroll
          for (int pp = 0; pp < HP; ++pp) ab[c][pp] = v[pp] + x8[pp];
        }
        publish();
        issue(tm + TG, tm + TD, sA, sAl, 16384, NC / 8, IDW);    // dW_l = zbar_l a_{l-1}^T
        wait_mma();
        {
          float* const gw = g + sh.woff[l] + (size_t)nrn * W + hf * 64;
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            float v[32], x[32];
            tc::ld32(tm + lrow + TG + (uint32_t)(hf * 64 + h2 * 32), v);
            tc::ld32(tm + lrow + TD + (uint32_t)(hf * 64 + h2 * 32), x);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              float4* const p4 = reinterpret_cast<float4*>(gw + h2 * 32 + j);
              float4 o = make_float4(v[j] + x[j], v[j + 1] + x[j + 1], v[j + 2] + x[j + 2], v[j + 3] + x[j + 3]);
              if (!first) {
                const float4 q = *p4;
                o.x += q.x; o.y += q.y; o.z += q.z; o.w += q.w;
              }
              *p4 = o;
            }
          }
        }
      }
      // first affine map: dW_0[i][q] += sum_p (zbar_val xh_q + s_q zbar_q), db_0
      {
        float part[DIN + 1];
#pragma unroll
        for (int q = 0; q <= DIN; ++q) part[q] = 0.f;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float hs[C][4];
          stash_ld4(0, j, hs);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float hz[C], av[C], zz[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
              hz[c] = hs[c][u];
              av[c] = ab[c][4 * j + u];
            }
            act_bwd<C, DS, DIN, ACT>(hz, av, zz);
            const int p = hf * HP + 4 * j + u;
#pragma unroll
            for (int q = 0; q < DIN; ++q) {
              part[q] = fmaf(zz[0], xh[p * 4 + q], part[q]);
              part[q] = fmaf(s_scale[q], zz[1 + q], part[q]);
            }
            part[DIN] += zz[0];
          }
        }
#pragma unroll
        for (int q = 0; q <= DIN; ++q) xpart[(hf * W + nrn) * 8 + q] = part[q];
      }
      __syncthreads();
      if (hf == 0) {
#pragma unroll
        for (int q = 0; q < DIN; ++q)
          grad_rmw(g + sh.woff[0] + nrn * DIN + q, xpart[nrn * 8 + q] + xpart[(W + nrn) * 8 + q], first);
        grad_rmw(g + sh.boff[0] + nrn, xpart[nrn * 8 + DIN] + xpart[(W + nrn) * 8 + DIN], first);
      }
      __syncthreads();
    }   // sub-tiles
    if (t == 0) {
      double* lp = b.loss_part + (size_t)item.slot * 5;
      for (int q = 0; q < 5; ++q) lp[q] = 0.0;
      lp[1] = lsum0;
    }
  }   // items
  // drain: after a time-out, give the outstanding MMAs a bounded time before
  // the tensor memory is released
  if (t == 0 && s_abort) mbar_wait_ok(&mbar, (phase + 1) & 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::dealloc(tm, TCOLS);
}

}  // namespace dk

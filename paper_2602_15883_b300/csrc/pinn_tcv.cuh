// Tensor-core (tcgen05, 3xTF32) variant of the value kernels for width 128:
// k_pinn<128, DS, UNST, false, MODE, ACT> for MODE = M_TRAIN (observation
// items, L_obs of Eq. (3), and the ghost terms of Eqs. (13)-(15) on face
// items, with the reverse pass), MODE = M_EVAL (the exchange of
// Algorithm 1: both sides' (u, p) at the face points and the masters'
// p(x_anc, t)) and MODE = M_QUERY (routed query points, with the anchored
// pressure of Eq. (18) by a second pass at x_anc for master nets).  Values
// only (one channel), 64 points per tile; the hidden contractions run as in
// k_pinn_tc (operands split into TF32 hi/lo, main and correction products in
// separate accumulators):
//
//   forward       Z_l       = W_l     a_{l-1}     M = 128 neurons, N = 64 points, K = 128
//   input adjoint abar_{l-1} = W_l^T  zbar_l      M = 128,         N = 64,        K = 128
//   weight grad   dW_l      = zbar_l  a_{l-1}^T   M = 128,         N = 128,       K = 64
//
// 512 threads; thread (warp w, lane) owns neuron 32 (w % 4) + lane and the
// points 16 (w / 4) .. + 15 of the tile.  Tensor memory as in k_pinn_tc
// (A operand hi/lo in [0, 256), accumulators at 256 and 384); shared memory:
// the [n][neuron] operand (32 KB hi + 32 KB lo) and the [neuron][n] operand
// (same), each of which doubles as the staging area of the next weight
// matrix while the other is in use.
#pragma once
#include "pinn_tc.cuh"

namespace dk {

struct TcvTile {
  static constexpr int W = 128;
  static constexpr int P = 64;                        // points per tile = columns
  static constexpr int NQ = NTC / 128;                // point groups (threads per neuron)
  static constexpr int HP = P / NQ;                   // points per thread
  static constexpr uint32_t XT = (uint32_t)P * 512;   // one [P][128] tile (hi or lo), bytes
  static constexpr uint32_t ABT = (uint32_t)(P / 32) * 16384;   // one [128][P] tile (hi or lo)
  static constexpr uint32_t R1 = 2 * XT;
  static constexpr uint32_t SMALL = R1 + 2 * ABT;
  static constexpr int RSO = P + 4;                   // row stride of a_{L-1} (FP32)
  static_assert(HP == 16, "16 points per thread");
  static_assert((size_t)W * RSO * 4 <= 2 * (size_t)ABT, "a_{L-1} buffer");
  static_assert((size_t)W * W * 4 <= 2 * (size_t)XT && (size_t)W * W * 4 <= 2 * (size_t)ABT, "weight staging");
};

template <int DOUT>
constexpr size_t tcv_smem_bytes(int L) {
  using T = TcvTile;
  return 1024 + T::SMALL +
         4 * ((size_t)2 * DOUT * T::P + T::P * 4 + T::W * 4 + T::W + DOUT * T::W + 4 + T::NQ * T::W * 8 +
              (size_t)(L > 1 ? L - 1 : 0) * T::W);
}

// stash floats per CTA: per layer and thread 16 values (4 float4)
constexpr long long tcv_stash_floats(int L) { return (long long)L * 4 * NTC * 4; }

template <int DS, int UNST, int ACT, int MODE>
__global__ void __launch_bounds__(NTC, 1)
    k_pinn_tcv(const Shape sh, const Bufs b, const Item* __restrict__ items, const int* __restrict__ n_items_ptr) {
  constexpr int W = 128, DIN = DS + UNST, DOUT = DS + 1;
  using T = TcvTile;
  constexpr int P = T::P, HP = T::HP, NQ = T::NQ, RSO = T::RSO;
  constexpr int KQ = W / NQ;
  constexpr uint32_t XT = T::XT, ABT = T::ABT;
  constexpr uint32_t IDN = tc::idesc_tf32(128, P), IDW = tc::idesc_tf32(128, 128);
  constexpr uint32_t TLO = 128, TD = 256, TG = 384, TCOLS = 512;
  constexpr bool TRAIN = (MODE == M_TRAIN);

  // Algorithm 1: the messages are refreshed every I_comm iterations and the
  // cached (stale) ones are used in between.
  if (MODE == M_EVAL && b.comm_interval > 1 && (*b.step % b.comm_interval) != 0) return;

  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t* const sb = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* const gX = sb;
  uint8_t* const gXl = sb + XT;
  uint8_t* const gA = sb + T::R1;
  uint8_t* const gAl = gA + ABT;
  const uint32_t sX = tc::saddr(gX), sXl = tc::saddr(gXl), sA = tc::saddr(gA), sAl = tc::saddr(gAl);
  float* const outa = reinterpret_cast<float*>(gA);             // a_{L-1} in FP32 [W][RSO]
  float* const ysm = reinterpret_cast<float*>(sb + T::SMALL);   // [DOUT][P]
  float* const ybsm = ysm + DOUT * P;
  float* const xh = ybsm + DOUT * P;      // [P][4]
  float* const w0s = xh + P * 4;          // [W][4]
  float* const b0s = w0s + W * 4;         // [W]
  float* const wLs = b0s + W;             // [DOUT][W]
  float* const bLs = wLs + DOUT * W;      // [4]
  float* const xpart = bLs + 4;           // [NQ][W][8]
  float* const bls = xpart + NQ * W * 8;  // [L-1][W]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t wbar;
  __shared__ __align__(8) uint64_t dbar;   // drain after a time-out
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort, s_other_master, s_is_time;
  __shared__ float s_red[NTC / 32];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int qd = warp & 3, hq = warp >> 2;
  const int nrn = qd * 32 + lane;
  const int p0 = hq * HP;
  const uint32_t lrow = (uint32_t)(qd * 32) << 16;
  const int L = sh.L;
  const int n_items = *n_items_ptr;

  if (t == 0) {
    mbar_init(&mbar, 1);
    mbar_init(&wbar, 1);
    mbar_init(&dbar, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::alloc(&s_tmem, TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = s_tmem;
  uint32_t phase = 0, wphase = 0;
  float4* const stash = reinterpret_cast<float4*>(b.stash + (TRAIN ? (size_t)blockIdx.x * b.stash_per_cta : 0));

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
  auto publish = [&]() {
    tc::wait_st();
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  };
  // stash: 4 float4 per layer (the thread's 16 points)
  auto stash_st = [&](int l, const float (&h)[HP]) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      stash[((size_t)l * 4 + j) * NTC + t] = make_float4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
  };
  auto stash_ld = [&](int l, float (&h)[HP]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = stash[((size_t)l * 4 + j) * NTC + t];
      h[4 * j] = v.x; h[4 * j + 1] = v.y; h[4 * j + 2] = v.z; h[4 * j + 3] = v.w;
    }
  };
  auto act = [&](float h) {
    if constexpr (ACT == ACT_SIN) {
      float sn, cs;
      sincos_act(h, &sn, &cs);
      return sn;
    } else {
      return h;
    }
  };
  auto put_row = [&](int u, float v) {   // point p0 + u, neuron nrn -> [n][neuron]
    const int n = p0 + u;
    const uint32_t off = (uint32_t)qd * (P * 128) + (uint32_t)(n >> 3) * 1024 + (uint32_t)(n & 7) * 128 +
                         ((uint32_t)((lane >> 2) ^ (n & 7)) << 4) + (uint32_t)(lane & 3) * 4;
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    *reinterpret_cast<float*>(gX + off) = hi;
    *reinterpret_cast<float*>(gXl + off) = lo;
  };
  auto put_col4 = [&](int j, float v0, float v1, float v2, float v3) {   // points p0 + 4 j .. + 3
    const int chunk = (hq & 1) * 4 + j;
    const uint32_t off = (uint32_t)(hq >> 1) * 16384 + (uint32_t)(nrn >> 3) * 1024 + (uint32_t)(nrn & 7) * 128 +
                         ((uint32_t)(chunk ^ (nrn & 7)) << 4);
    float4 h4, l4;
    tc::split_tf32(v0, h4.x, l4.x);
    tc::split_tf32(v1, h4.y, l4.y);
    tc::split_tf32(v2, h4.z, l4.z);
    tc::split_tf32(v3, h4.w, l4.w);
    *reinterpret_cast<float4*>(gA + off) = h4;
    *reinterpret_cast<float4*>(gAl + off) = l4;
  };
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
  auto put_w_staged = [&](const float* ws) {
    mbar_wait(&wbar, wphase & 1, b.err);
    ++wphase;
    float hi[KQ], lo[KQ];
#pragma unroll
    for (int j = 0; j < KQ; ++j) tc::split_tf32(ws[(hq * KQ + j) * W + nrn], hi[j], lo[j]);
    tc::st32(tm + lrow + (uint32_t)(hq * KQ), hi);
    tc::st32(tm + lrow + TLO + (uint32_t)(hq * KQ), lo);
  };
  auto put_act = [&](int l, const float (&h)[HP]) {   // activations of the thread's points
    if (l + 1 < L) {
#pragma unroll
      for (int u = 0; u < HP; ++u) put_row(u, act(h[u]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4*>(outa + nrn * RSO + p0 + 4 * j) =
            make_float4(act(h[4 * j]), act(h[4 * j + 1]), act(h[4 * j + 2]), act(h[4 * j + 3]));
    }
  };
  auto ld_result = [&](float (&r)[HP]) {
    float v[16], x[16];
    tc::ld16_pair(tm + lrow + TD + (uint32_t)p0, tm + lrow + TG + (uint32_t)p0, v, x);
#pragma unroll
    for (int u = 0; u < HP; ++u) r[u] = v[u] + x[u];
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
    double lsum0 = 0.0, lsum1 = 0.0;   // thread 0: loss numerators of the item
    const int npass = (MODE == M_QUERY && ni.master) ? 2 : 1;

    for (int sub = 0; sub < item.count; sub += P) {
      const int npts = min(P, item.count - sub);
      const bool first = (sub == 0);
      float pkeep = 0.f;   // query: raw pressure of a master point (thread t = point)
     for (int pass = 0; pass < npass; ++pass) {
      // ---- inputs mapped to the net's box
      if (t < P) {
        const bool valid = t < npts;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid) {
          const float* src =
              MODE == M_QUERY ? b.q_pts + (size_t)b.q_perm[item.begin + sub + t] * DIN
                              : (item.kind == K_OBS ? b.obs_pts : b.face_pts) + (size_t)(item.begin + sub + t) * DIN;
#pragma unroll
          for (int q = 0; q < DIN; ++q) x[q] = src[q];
          if (item.kind == K_EVAL_ANC || pass == 1) {   // p(x_anc, t) at the point's time, Eqs. (15), (18)
#pragma unroll
            for (int q = 0; q < DS; ++q) x[q] = sh.anchor[q];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) xh[t * 4 + q] = (valid && q < DIN) ? (x[q] - ni.center[q]) * ni.scale[q] : 0.f;
      }
      __syncthreads();
      // ---- first affine map (FP32)
      {
        float w[DIN];
#pragma unroll
        for (int q = 0; q < DIN; ++q) w[q] = w0s[nrn * 4 + q];
        const float bias = b0s[nrn];
        float h[HP];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float v = bias;
#pragma unroll
          for (int q = 0; q < DIN; ++q) v = fmaf(w[q], xh[(p0 + u) * 4 + q], v);
          h[u] = stash_value<ACT>(v);
        }
        if (TRAIN) stash_st(0, h);
        put_act(0, h);
      }
      // ---- hidden layers on the tensor cores
      if (L > 1) put_w(th + sh.woff[1] + (size_t)nrn * W + hq * KQ);
      for (int l = 1; l < L; ++l) {
        publish();
        issue(tm + TD, tm + TG, sX, sXl, P * 128, W / 8, IDN);
        if (t == 0 && l + 1 < L) bulk_load(gA, thT + (size_t)l * W * W, W * W * 4, &wbar);
        wait_mma();
        float h[HP];
        ld_result(h);
        if (l + 1 < L) put_w_staged(reinterpret_cast<const float*>(gA));
        const float bias = bls[(l - 1) * W + nrn];
#pragma unroll
        for (int u = 0; u < HP; ++u) h[u] = stash_value<ACT>(h[u] + bias);
        if (TRAIN) stash_st(l, h);
        put_act(l, h);
      }
      __syncthreads();
      // ---- output layer (FP32): Y[j][p] = W_L[j] . a_{L-1}[.][p] + b_L[j]
      {
        constexpr int PAIRS = DOUT * P;
        constexpr int KS = NTC / PAIRS >= 2 ? 2 : 1;
        for (int pr = t / KS; pr < PAIRS; pr += NTC / KS) {
          const int j = pr / P, p = pr % P, lk = t % KS;
          float acc = 0.f;
          for (int k = lk; k < W; k += KS) acc = fmaf(wLs[j * W + k], outa[k * RSO + p], acc);
          if (KS == 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (lk == 0) ysm[j * P + p] = acc + bLs[j];
        }
      }
      __syncthreads();
      // ---- per-point epilogue (thread = point)
      float l0 = 0.f, l1 = 0.f;
      if (t < P) {
        const bool valid = t < npts;
        const size_t pt = (size_t)(item.begin + sub + t);
        float Y[DOUT];
#pragma unroll
        for (int j = 0; j < DOUT; ++j) Y[j] = ysm[j * P + t];
        if constexpr (TRAIN) {
          float Yb[DOUT];
#pragma unroll
          for (int j = 0; j < DOUT; ++j) Yb[j] = 0.f;
          if (valid && item.kind == K_OBS) {   // Eq. (3)
            const float* ov = b.obs_vals + pt * DS;
#pragma unroll
            for (int c = 0; c < DS; ++c) {
              const float e = Y[c] - ov[c];
              l0 = fmaf(sh.comp_w[c] * e, e, l0);
              Yb[c] = 2.f * sh.lam_obs * sh.comp_w[c] * e * ni.inv_nobs;
            }
          } else if (valid) {   // K_FACE, Eqs. (13)-(15)
            const int o = 1 - item.side;
            const float* nv = b.nbr_val + (pt * 2 + o) * DOUT;
#pragma unroll
            for (int c = 0; c < DS; ++c) {
              const float e = Y[c] - nv[c];
              l0 = fmaf(sh.comp_w[c] * e, e, l0);
              Yb[c] = 2.f * sh.lam_gh_u * sh.comp_w[c] * e * ni.inv_ngh;
            }
            float Pn = nv[DS];
            if (s_other_master) Pn = Pn - b.nbr_anc[pt * 2 + o];
            const float ep = Y[DS] - Pn;
            const float lam = s_is_time ? sh.lam_time : ni.lam_space;
            Yb[DS] = 2.f * lam * ep * ni.inv_ngh;
            l1 = ep * ep;
          }
#pragma unroll
          for (int j = 0; j < DOUT; ++j) ybsm[j * P + t] = Yb[j];
        } else if (MODE == M_QUERY) {
          if (valid) {
            float* o = b.q_out + (size_t)b.q_perm[item.begin + sub + t] * b.q_w;
            if (pass == 0) {
#pragma unroll
              for (int j = 0; j < DS; ++j) o[j] = Y[j];
              if (npass == 1) o[DS] = Y[DS] + sh.p_ref;
              else pkeep = Y[DS];
            } else {
              o[DS] = (pkeep - Y[DS]) + sh.p_ref;
            }
          }
        } else if (valid) {
          if (item.kind == K_EVAL) {
#pragma unroll
            for (int j = 0; j < DOUT; ++j) b.nbr_val[(pt * 2 + item.side) * DOUT + j] = Y[j];
          } else {
            b.nbr_anc[pt * 2 + item.side] = Y[DS];
          }
        }
      }
      if constexpr (TRAIN) {
        const float s0 = block_sum_tc(l0, s_red);
        if (t == 0) lsum0 += (double)s0;
        if (item.kind == K_FACE) {
          const float s1 = block_sum_tc(l1, s_red);
          if (t == 0) lsum1 += (double)s1;
        }
      }
      __syncthreads();
     }   // pass
      if constexpr (!TRAIN) continue;
      if (b.no_reverse) continue;

      // ================= reverse pass =================
      float* const g = b.grad_part + (size_t)item.slot * sh.npp;
      float hsn[HP];
      stash_ld(L - 1, hsn);
      if (L > 1) put_w(thT + (size_t)(L - 2) * W * W + (size_t)nrn * W + hq * KQ);
      for (int e = t; e < DOUT * W; e += NTC) {   // dW_L, from a_{L-1} (FP32) and the seeds
        const int j = e / W, k = e % W;
        float s = 0.f;
        for (int p = 0; p < P; ++p) s = fmaf(ybsm[j * P + p], outa[k * RSO + p], s);
        gacc(g + sh.woff[L] + e, s, first);
      }
      if (t < DOUT) {
        float s = 0.f;
        for (int p = 0; p < P; ++p) s += ybsm[t * P + p];
        gacc(g + sh.boff[L] + t, s, first);
      }
      float ab[HP];
      {
        float wl[DOUT];
#pragma unroll
        for (int j = 0; j < DOUT; ++j) wl[j] = wLs[j * W + nrn];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float v = 0.f;
#pragma unroll
          for (int j = 0; j < DOUT; ++j) v = fmaf(wl[j], ybsm[j * P + p0 + u], v);
          ab[u] = v;
        }
      }
      for (int l = L - 1; l >= 1; --l) {
        float zb[HP];
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float zz;
          act_bwd<1, DS, DIN, ACT>(&hsn[u], &ab[u], &zz);
          zb[u] = zz;
        }
        {
          float s = 0.f;
#pragma unroll
          for (int u = 0; u < HP; ++u) s += zb[u];
          xpart[(hq * W + nrn) * 8] = s;
        }
#pragma unroll
        for (int u = 0; u < HP; ++u) put_row(u, zb[u]);
        if (t == 0) bulk_flush_wait();   // the previous layer's tile has left the staging region
        publish();
        issue(tm + TD, tm + TG, sX, sXl, P * 128, W / 8, IDN);   // abar_{l-1} = W_l^T zbar_l
        stash_ld(l - 1, hsn);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          put_col4(j, act(hsn[4 * j]), act(hsn[4 * j + 1]), act(hsn[4 * j + 2]), act(hsn[4 * j + 3]));
        if (hq == 0) {
          float s = 0.f;
#pragma unroll
          for (int q = 0; q < NQ; ++q) s += xpart[(q * W + nrn) * 8];
          gacc(g + sh.boff[l] + nrn, s, first);
        }
        wait_mma();
        if (t == 0 && l > 1) bulk_load(gX, th + sh.woff[l - 1], W * W * 4, &wbar);
        {   // zbar_l -> tensor memory (A operand of the weight gradient)
          float hv[16], lv[16];
#pragma unroll
          for (int u = 0; u < HP; ++u) tc::split_tf32(zb[u], hv[u], lv[u]);
          tc::st16(tm + lrow + (uint32_t)p0, hv);
          tc::st16(tm + lrow + TLO + (uint32_t)p0, lv);
        }
        ld_result(ab);
        publish();
        issue(tm + TG, tm + TD, sA, sAl, 16384, P / 8, IDW);    // dW_l = zbar_l a_{l-1}^T
        wait_mma();
        {
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
          // staged row-major in the idle [neuron][n] operand region, one
          // 128-byte row segment per group of 8 lanes
          const int row0 = qd * 32 + (lane & ~7);
          float* const sw = reinterpret_cast<float*>(gA) + row0 * W + hq * KQ + 4 * (lane & 7);
#pragma unroll
          for (int c = 0; c < 8; ++c) *reinterpret_cast<float4*>(sw + c * W) = q[c];
          tc::fence_smem_async();
        }
        if (l > 1) put_w_staged(reinterpret_cast<const float*>(gX));
        __syncthreads();
        if (t == 0) bulk_flush(g + sh.woff[l], sA, W * W * 4, first);
      }
      // first affine map: dW_0[i][q] += sum_p zbar_p xh_{p,q}, db_0
      {
        float part[DIN + 1];
#pragma unroll
        for (int q = 0; q <= DIN; ++q) part[q] = 0.f;
#pragma unroll
        for (int u = 0; u < HP; ++u) {
          float zz;
          act_bwd<1, DS, DIN, ACT>(&hsn[u], &ab[u], &zz);
#pragma unroll
          for (int q = 0; q < DIN; ++q) part[q] = fmaf(zz, xh[(p0 + u) * 4 + q], part[q]);
          part[DIN] += zz;
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
      if (item.kind == K_OBS) lp[0] = lsum0;
      else {
        lp[2] = lsum0;
        lp[s_is_time ? 4 : 3] = lsum1;
      }
    }
  }   // items
  // drain after a time-out: mbar's parity is unknown once waits were skipped,
  // so a commit to a barrier of its own tracks every MMA issued before it
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

// Non-template kernels of libdpinn (sm_103a): deterministic gradient
// reduction, optional clipping and Adam, the loss record, the query router
// and parameter initialisation.  Included by the host runtime only (the
// grouped kernel templates live in pinn_kernels.cuh).
#pragma once
#include "pinn_kernels.cuh"

namespace dk {

// ----------------------------------------------- reduction + Adam ---
// grad[k][j] = sum over the work items of net k (fixed order); per-block
// partial squared norms for clipping.
__global__ void k_reduce_grad(const float* __restrict__ part, const int* __restrict__ slot_begin,
                              float* __restrict__ grad, float* __restrict__ norm_part, int npp, int n_params) {
  __shared__ float red[NT / 32];
  const int k = blockIdx.y;
  const int j = blockIdx.x * NT + threadIdx.x;
  float gsum = 0.f;
  if (j < n_params) {
    const int s0 = slot_begin[k], s1 = slot_begin[k + 1];
    for (int s = s0; s < s1; ++s) gsum += part[(size_t)s * npp + j];
    grad[(size_t)k * npp + j] = gsum;
  }
  const float tot = block_sum(gsum * gsum, red);
  if (threadIdx.x == 0) norm_part[(size_t)k * gridDim.x + blockIdx.x] = tot;
}

// Per-net clip coefficient min(1, clip / (||g|| + 1e-6)), fixed-order sum.
__global__ void k_clip_coef(const float* __restrict__ norm_part, int nblk, float clip, float* __restrict__ coef) {
  __shared__ float red[NT / 32];
  const int k = blockIdx.x;
  float s = 0.f;
  for (int i = threadIdx.x; i < nblk; i += NT) s += norm_part[(size_t)k * nblk + i];
  const float tot = block_sum(s, red);
  if (threadIdx.x == 0) {
    const float c = clip / (sqrtf(tot) + 1e-6f);
    coef[k] = c < 1.f ? c : 1.f;
  }
}

struct AdamArgs {
  double lr, beta1, beta2, eps;
  int use_clip;
  double decay_factor;   // lr * decay_factor^floor((t-1)/decay_interval)
  int decay_interval;    // 0: constant lr
  // log(beta1), log(beta2), log(decay_factor), formed in double on the host:
  // the bias corrections 1 - beta^t = -expm1(t log beta) then take a few FP32
  // operations with about 1e-7 relative error (1 - 0.999^t included), where
  // FP64 pow on every block cost more than the update itself
  float log_beta1, log_beta2, log_decay;
};
// (1 - beta) factors are formed in double on the host and rounded once:
// 1.f - 0.999f would carry a 1.3e-5 relative error into the second moment.

// Adam (PyTorch's rule) on every parameter of every net; rewrites the
// transposed copies of the hidden weights used by the forward pass.
__global__ void k_adam(const Shape sh, AdamArgs ar, float* __restrict__ theta, float* __restrict__ thetaT,
                       float* __restrict__ m, float* __restrict__ v, const float* __restrict__ grad,
                       const float* __restrict__ coef, const long long* __restrict__ step, int n_params) {
  __shared__ float s_c[4];
  if (threadIdx.x == 0) {
    const float t = (float)(*step + 1);
    const float bc1 = -expm1f(t * ar.log_beta1);
    const float bc2 = -expm1f(t * ar.log_beta2);
    float lr = (float)ar.lr;
    if (ar.decay_interval > 0) {
      const long long n = (*step) / ar.decay_interval;
      if (n > 0) lr *= expf((float)n * ar.log_decay);
    }
    s_c[0] = lr / bc1;
    s_c[1] = 1.f / sqrtf(bc2);
  }
  __syncthreads();
  const int k = blockIdx.y;
  const int j = blockIdx.x * NT + threadIdx.x;
  if (j >= n_params) return;
  const size_t idx = (size_t)k * sh.npp + j;
  float gj = grad[idx];
  if (ar.use_clip) gj *= coef[k];
  const float b1 = (float)ar.beta1, b2 = (float)ar.beta2;
  const float omb1 = (float)(1.0 - ar.beta1), omb2 = (float)(1.0 - ar.beta2);
  const float mj = fmaf(b1, m[idx], omb1 * gj);
  const float vj = fmaf(b2, v[idx], omb2 * gj * gj);
  m[idx] = mj;
  v[idx] = vj;
  const float denom = sqrtf(vj) * s_c[1] + (float)ar.eps;
  const float th = theta[idx] - s_c[0] * (mj / denom);
  theta[idx] = th;
  const int W = sh.W;
  for (int l = 1; l < sh.L; ++l) {
    if (j >= sh.woff[l] && j < sh.boff[l]) {
      const int r = j - sh.woff[l], i = r / W, c = r % W;
      if (sh.twp == 0) {
        thetaT[(size_t)k * sh.nTp + (size_t)(l - 1) * W * W + (size_t)c * W + i] = th;
      } else {   // streamed-weight layout: forward block row c, reverse block row i
        float* const tl = thetaT + (size_t)k * sh.nTp + (size_t)(l - 1) * 2 * W * sh.twp;
        tl[(size_t)c * sh.twp + wide_pos(i, sh.twp)] = th;
        tl[(size_t)(W + i) * sh.twp + wide_pos(c, sh.twp)] = th;
      }
    }
  }
}

// Rebuild the transposed hidden weights from theta (after set_state/init).
// The streamed-weight layout is written whole, its padded entries as zeros
// (k_adam rewrites only the others).
__global__ void k_transpose(const Shape sh, const float* __restrict__ theta, float* __restrict__ thetaT) {
  const int k = blockIdx.y;
  const int W = sh.W;
  const int e = blockIdx.x * NT + threadIdx.x;
  const float* const th = theta + (size_t)k * sh.npp;
  if (sh.twp == 0) {
    if (e >= (sh.L - 1) * W * W) return;
    const int l = 1 + e / (W * W), r = e % (W * W), i = r / W, c = r % W;
    thetaT[(size_t)k * sh.nTp + (size_t)(l - 1) * W * W + (size_t)c * W + i] = th[sh.woff[l] + r];
  } else {
    const int WP = sh.twp;
    if (e >= (sh.L - 1) * 2 * W * WP) return;
    const int l = 1 + e / (2 * W * WP), r = e % (2 * W * WP), row = r / WP, n = r % WP;
    float v = 0.f;
    if (n < W) v = (row < W) ? th[sh.woff[l] + n * W + row]           // forward: W_l^T[row][n]
                             : th[sh.woff[l] + (row - W) * W + n];    // reverse: W_l[row - W][n]
    thetaT[(size_t)k * sh.nTp + (size_t)(l - 1) * 2 * W * WP + (size_t)row * WP + wide_pos(n, WP)] = v;
  }
}

// Loss record per net: fixed-order sum of the item partials, 1/N factors,
// weighted total (Eq. (16)); non-finite values raise ERR_NONFINITE.
__global__ void k_loss_record(const Shape sh, const double* __restrict__ loss_part, const int* __restrict__ slot_begin,
                              const NetInfo* __restrict__ nets, int n_nets, float* __restrict__ rec, int* err,
                              long long* step, int bump) {
  // one warp per net: lane j sums slots j, j + 32, ... in order, then a
  // fixed shuffle tree; lane 0's total is the recorded value
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0 && bump) *step += 1;
  if (k >= n_nets) return;
  double s[LP] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = slot_begin[k] + lane; i < slot_begin[k + 1]; i += 32)
#pragma unroll
    for (int q = 0; q < LP; ++q) s[q] += loss_part[(size_t)i * LP + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < LP; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
  if (lane != 0) return;
  const NetInfo ni = nets[k];
  const double lo = s[0] * ni.inv_nobs, lp = s[1] * ni.inv_npde, lu = s[2] * ni.inv_ngh,
               ls = s[3] * ni.inv_ngh, lt = s[4] * ni.inv_ngh, lr = s[5] * ni.inv_ngh, lc = s[6] * ni.inv_ngh;
  const double tot = sh.lam_obs * lo + sh.lam_pde * lp + sh.lam_gh_u * lu + ni.lam_space * ls + sh.lam_time * lt +
                     sh.lam_gh_r * lr + sh.lam_gh_c1 * lc;
  const double v[8] = {lo, lp, lu, ls, lt, tot, lr, lc};
  for (int q = 0; q < 8; ++q) {
    rec[k * 8 + q] = (float)v[q];
    if (!isfinite(v[q])) atomicExch(err + ERR_NONFINITE, 1);
  }
}

// ----------------------------------------------------------- routing ---
struct Route {
  float lo[4], hi[4], inv_h[4];
  int splits[4], stride[4];
  int din, n_nets;
};

// Cell of every query point (float32 rule of the C ABI) and per-net counts.
__global__ void k_route(const Route rt, const float* __restrict__ pts, long long n, int* __restrict__ net_of,
                        int* __restrict__ counts, int* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int net = 0;
  bool ok = true;
  for (int a = 0; a < rt.din; ++a) {
    const float x = pts[i * rt.din + a];
    if (!(x >= rt.lo[a] && x <= rt.hi[a])) { ok = false; break; }
    const float q = __fmul_rn(__fsub_rn(x, rt.lo[a]), rt.inv_h[a]);
    int c = (int)floorf(q);
    c = c < 0 ? 0 : (c > rt.splits[a] - 1 ? rt.splits[a] - 1 : c);
    net += c * rt.stride[a];
  }
  if (!ok) {
    net_of[i] = -1;
    atomicExch(err + ERR_DOMAIN, 1);
    return;
  }
  net_of[i] = net;
  atomicAdd(counts + net, 1);
}

// Single block: segment offsets per net and the query work items (chunks of
// `chunk` points); cursor[] starts at the offsets for the scatter.
__global__ void k_route_plan(const int* __restrict__ counts, int n_nets, int chunk, int* __restrict__ offsets,
                             int* __restrict__ cursor, Item* __restrict__ items, int* __restrict__ n_items) {
  if (threadIdx.x != 0) return;
  int off = 0, ni = 0;
  for (int k = 0; k < n_nets; ++k) {
    offsets[k] = off;
    cursor[k] = off;
    const int c = counts[k];
    for (int s = 0; s < c; s += chunk) {
      Item it;
      it.kind = K_QUERY; it.net = k; it.begin = off + s; it.count = min(chunk, c - s);
      it.slot = 0; it.face = 0; it.side = 0; it.pad = 0;
      items[ni++] = it;
    }
    off += c;
  }
  *n_items = ni;
}

__global__ void k_route_scatter(const int* __restrict__ net_of, long long n, int* __restrict__ cursor,
                                int* __restrict__ perm) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = net_of[i];
  if (k < 0) return;
  perm[atomicAdd(cursor + k, 1)] = (int)i;
}

// --------------------------------------------------- initialisation ---
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Xavier-normal weights (std sqrt(2/(fan_in+fan_out))), zero biases; normal
// deviates by Box-Muller from a SplitMix64 counter stream keyed by
// (seed, net, parameter index).
__global__ void k_init(const Shape sh, uint64_t seed, float* __restrict__ theta, int n_params) {
  const int k = blockIdx.y;
  const int j = blockIdx.x * NT + threadIdx.x;
  if (j >= n_params) return;
  float val = 0.f;
  for (int l = 0; l <= sh.L; ++l) {
    const int fo = (l == sh.L) ? sh.dout : sh.W;
    const int fi = (l == 0) ? sh.din : sh.W;
    if (j >= sh.woff[l] && j < sh.boff[l]) {
      const uint64_t key = splitmix64(seed ^ splitmix64(((uint64_t)k << 32) | (uint64_t)j));
      const uint64_t r2 = splitmix64(key);
      const double u1 = ((key >> 11) + 1.0) * (1.0 / 9007199254740993.0);
      const double u2 = (r2 >> 11) * (1.0 / 9007199254740992.0);
      const double nrm = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      val = (float)(nrm * sqrt(2.0 / (fi + fo)));
    }
  }
  theta[(size_t)k * sh.npp + j] = val;
}

// ---- per-step resampling of the collocation points --------------------
// SplitMix64 (Steele, Lea and Flood, 2014): the n-th output (n = 1, 2, ...) of
// the generator seeded with S is mix(S + n * gamma).  Streams: S_t = the
// (t+1)-th output for the step seed, S_{t,k} = the (k+1)-th output of S_t for
// net k; coordinate d of point i uses output i * d_in + d + 1 of S_{t,k}, whose
// top 24 bits give u in [0, 1) exactly; x = lo + u * w in double (no fused
// multiply-add), rounded to float32.
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;

// grid.y = net; box[k] = {lo[4], w[4]} (double)
__global__ void k_sample(int din, uint64_t seed, const long long* __restrict__ step,
                         const long long* __restrict__ offsets, const double* __restrict__ box,
                         float* __restrict__ pts) {
  const int k = blockIdx.y;
  const long long n = offsets[k + 1] - offsets[k];
  const uint64_t st = sm64_mix(seed + (uint64_t)(*step + 1) * SM64_GAMMA);
  const uint64_t sk = sm64_mix(st + (uint64_t)(k + 1) * SM64_GAMMA);
  const double* lo = box + (size_t)k * 8;
  const double* w = lo + 4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float* out = pts + (offsets[k] + i) * din;
    for (int d = 0; d < din; ++d) {
      const uint64_t o = sm64_mix(sk + (uint64_t)(i * din + d + 1) * SM64_GAMMA);
      const double u = (double)(o >> 40) * (1.0 / 16777216.0);
      out[d] = __double2float_rn(__dadd_rn(lo[d], __dmul_rn(u, w[d])));
    }
  }
}

// Self-test of the sin activation's sine and cosine: out[2 i], out[2 i + 1]
// = sincos_act(x[i]).
__global__ void k_selftest_sincos(const float* __restrict__ x, long long n, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s, c;
    sincos_act(x[i], &s, &c);
    out[2 * i] = s;
    out[2 * i + 1] = c;
  }
}

// Self-test of the bounded device waits: an mbarrier that nothing ever
// completes.  mbar_wait gives up after about 2 s and raises ERR_TIMEOUT in
// `err`; the kernel then returns normally.
__global__ void k_selftest_wait(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  mbar_wait(&bar, 0, err);
}

}  // namespace dk

// Host runtime and C ABI of libdpinn (declarations and conventions in
// include/dpinn.h).
//
// The handle owns the decomposition (cells, faces, masters - Sec. 2.2 and
// Algorithm 1), every device buffer, the work lists of the grouped kernels
// and two captured CUDA graphs: one training step (neighbour exchange,
// grouped jet/value forward + loss + reverse, deterministic gradient
// reduction, Adam) and the same without the optimiser update.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dpinn.h"
#include "kernel_set.h"
#include "pinn_aux.cuh"

namespace {

using dk::KernelSet;

bool pick_kernels(int W, int ds, int unst, int L, int act, KernelSet* k) {
  const bool sn = (act == DPINN_ACT_SIN);
  if (W == 32) return sn ? dk::kernels_w32_sin(ds, unst, L, k) : dk::kernels_w32_tanh(ds, unst, L, k);
  if (W == 64) return sn ? dk::kernels_w64_sin(ds, unst, L, k) : dk::kernels_w64_tanh(ds, unst, L, k);
  if (W == 128) return sn ? dk::kernels_w128_sin(ds, unst, L, k) : dk::kernels_w128_tanh(ds, unst, L, k);
  if (W > 128 && W <= 160) return sn ? dk::kernels_wide160_sin(ds, unst, L, k) : dk::kernels_wide160_tanh(ds, unst, L, k);
  if (W > 160 && W <= 224) return sn ? dk::kernels_wide224_sin(ds, unst, L, k) : dk::kernels_wide224_tanh(ds, unst, L, k);
  return false;
}

// float32 cell rule of the C ABI
int cell_fp32(const dpinn_config& c, int a, float x) {
  const float lo = (float)c.lo[a], hi = (float)c.hi[a];
  const float inv_h = (float)((double)c.splits[a] / (c.hi[a] - c.lo[a]));
  if (!(x >= lo && x <= hi)) return -1;
  volatile float d = x - lo;
  volatile float q = d * inv_h;
  int k = (int)std::floor((float)q);
  return std::min(std::max(k, 0), c.splits[a] - 1);
}

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  void free_() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t cnt) {
    if (cnt <= n && p) return cudaSuccess;
    free_();
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(cnt, 1) * sizeof(T));
    if (e == cudaSuccess) n = std::max<size_t>(cnt, 1);
    else p = nullptr;
    return e;
  }
};

}  // namespace

struct dpinn {
  dpinn_config cfg{};
  int ds = 0, unst = 0, din = 0, dout = 0, W = 0, L = 0;
  int n_nets = 0, n_faces = 0, n_params = 0, npp = 0, nTp = 0;
  std::vector<int> stride, master;
  std::vector<std::array<int, 4>> cell;
  std::vector<std::array<double, 4>> blo, bhi;
  std::vector<std::array<int, 3>> faces;   // lo, hi, axis
  std::vector<std::vector<int>> net_faces; // face ids per net
  dk::Shape shape{};
  KernelSet ks;
  int dev = 0, n_sms = 0;
  int tile_jet = 0, tile_val = 0;   // FP32 point tiles: 0 default, 1 alternate
  std::string err;

  // parameters and optimiser state
  DevBuf<float> theta, thetaT, m, v, grad, norm_part, coef;
  DevBuf<long long> step_d;
  DevBuf<dk::NetInfo> nets_d;
  DevBuf<int> face_info_d, err_d, counters, n_items_d, slot_begin_d, iota_d;
  // points
  DevBuf<float> res_pts, obs_pts, obs_vals, face_pts;
  std::vector<int64_t> res_counts, obs_counts, face_counts;
  bool have[3] = {false, false, false};
  // per-step resampling of the residual points (dpinn_set_resampling)
  bool resample = false;
  uint64_t rs_seed = 0;
  int64_t rs_max = 0;
  DevBuf<long long> rs_off;
  DevBuf<double> rs_box;
  // gradient-partial memory budget (bytes) bounding the number of work items
  int64_t part_budget = (int64_t)1 << 30;
  // volumetric ghost layers: directed segments (own net, owner net, is_time)
  // of the ghost points, grouped by own net then owner
  bool ghost_mode = false;
  std::vector<std::array<int, 3>> seg;
  std::vector<int64_t> seg_counts;
  // plan
  DevBuf<dk::Item> items_eval, items_jet, items_val, items_jf;
  int n_eval = 0, n_jet = 0, n_val = 0, n_jf = 0, n_slots = 0;
  int grid_eval = 0, grid_jet = 0, grid_val = 0, grid_jf = 0;
  // interface residual / C1 terms on (face items train with jets)
  bool iface = false;
  // stash: the jet kernel's per-CTA activation stash; stash_side: the same for
  // the kernels of the step's side branch (face jets, values), which run
  // concurrently with the jet kernel
  DevBuf<float> grad_part, stash, stash_side, nbr_val, nbr_anc, nbr_res, nbr_grd, loss_rec;
  DevBuf<double> loss_part;
  float* loss_host = nullptr;
  bool plan_ok = false;
  int sched_jet = 0, sched_val = 0, sched_order = 0;   // 0 = automatic / longest first
  cudaStream_t cap = nullptr;
  // second capture stream: exchange, face-jet and value items fork off the
  // residual-point jet kernel (which needs no neighbour messages) and join
  // before the gradient reduction
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // asynchronous residual-point upload: host -> staging buffer on copy_st
  // (overlapping the running step), staging -> res_pts at the next launch
  cudaStream_t copy_st = nullptr;
  cudaEvent_t stage_ready = nullptr, stage_free = nullptr;
  DevBuf<float> res_stage;
  bool stage_pending = false;
  size_t stage_bytes = 0;
  cudaGraphExec_t g_step = nullptr, g_grad = nullptr, g_loss = nullptr;
  cudaEvent_t done = nullptr;
  int launches = 0;
  // query scratch
  DevBuf<int> q_net, q_perm, q_counts, q_off, q_cursor, q_nitems;
  DevBuf<dk::Item> q_items;

  ~dpinn() {
    if (g_step) cudaGraphExecDestroy(g_step);
    if (g_grad) cudaGraphExecDestroy(g_grad);
    if (g_loss) cudaGraphExecDestroy(g_loss);
    if (done) cudaEventDestroy(done);
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    if (stage_ready) cudaEventDestroy(stage_ready);
    if (stage_free) cudaEventDestroy(stage_free);
    if (copy_st) cudaStreamDestroy(copy_st);
    res_stage.free_();
    if (loss_host) cudaFreeHost(loss_host);
    for (auto* b : {&theta, &thetaT, &m, &v, &grad, &norm_part, &coef, &res_pts, &obs_pts, &obs_vals, &face_pts,
                    &grad_part, &stash, &stash_side, &nbr_val, &nbr_anc, &nbr_res, &nbr_grd, &loss_rec})
      b->free_();
    step_d.free_(); nets_d.free_(); loss_part.free_();
    for (auto* b : {&face_info_d, &err_d, &counters, &n_items_d, &slot_begin_d, &iota_d, &q_net, &q_perm,
                    &q_counts, &q_off, &q_cursor, &q_nitems})
      b->free_();
    items_eval.free_(); items_jet.free_(); items_val.free_(); items_jf.free_(); q_items.free_();
  }
};

namespace {

thread_local std::string g_create_err;

int fail(dpinn* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(dpinn* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? DPINN_ERR_OOM : DPINN_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

dk::Bufs make_bufs(dpinn* h) {
  dk::Bufs b{};
  b.theta = h->theta.p;
  b.thetaT = h->thetaT.p;
  b.nets = h->nets_d.p;
  b.res_pts = h->res_pts.p;
  b.obs_pts = h->obs_pts.p;
  b.obs_vals = h->obs_vals.p;
  b.face_pts = h->face_pts.p;
  b.face_info = h->face_info_d.p;
  b.nbr_val = h->nbr_val.p;
  b.nbr_anc = h->nbr_anc.p;
  b.nbr_res = h->nbr_res.p;
  b.nbr_grd = h->nbr_grd.p;
  b.grad_part = h->grad_part.p;
  b.loss_part = h->loss_part.p;
  b.stash = h->stash.p;
  b.stash_per_cta = 0;
  b.counter = h->counters.p;
  b.err = h->err_d.p;
  b.step = h->step_d.p;
  b.comm_interval = h->cfg.comm_interval;
  return b;
}

// Adam's arguments; the logarithms feed the FP32 bias corrections of k_adam
dk::AdamArgs adam_args(const dpinn* h) {
  const dpinn_config& c = h->cfg;
  return dk::AdamArgs{c.lr, c.beta1, c.beta2, c.eps, c.clip_norm > 0 ? 1 : 0, c.lr_decay_factor,
                      c.lr_decay_interval, (float)std::log(c.beta1), (float)std::log(c.beta2),
                      (float)std::log(c.lr_decay_factor)};
}

cudaError_t launch_pinn(const void* fn, int grid, size_t smem, const dk::Shape& sh, const dk::Bufs& b,
                        const dk::Item* items, const int* n_items, cudaStream_t s, int threads = dk::NT) {
  void* args[] = {(void*)&sh, (void*)&b, (void*)&items, (void*)&n_items};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

int occupancy(const void* fn, size_t smem, int threads = dk::NT) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess) return 1;
  return std::max(occ, 1);
}

// Split `count` points starting at `begin` into chunks of at most `chunk`.
template <class F>
void chunks(int64_t begin, int64_t count, int64_t chunk, F f) {
  for (int64_t s = 0; s < count; s += chunk) f(begin + s, std::min(chunk, count - s));
}

int build_plan(dpinn* h);

// Enqueue one step's work on stream s.  With `ev` (an array of at least 8
// events) an event is recorded before the first and after every kernel, and
// the kernel names are reported in `names` (for per-kernel timing).
// Step modes: the training step, gradients without the update, losses only.
enum { RUN_STEP = 0, RUN_GRAD = 1, RUN_LOSS = 2 };

// A training launch writes grid x stash_per_cta floats of its stash buffer:
// refuse (host side) any launch that the buffer does not cover.
static bool stash_fits(const DevBuf<float>& buf, int grid, long long per_cta) {
  return (size_t)std::max(grid, 0) * (size_t)std::max<long long>(per_cta, 0) <= buf.n;
}

cudaError_t enqueue_step(dpinn* h, int mode, cudaStream_t s, int* n_launch, cudaEvent_t* ev = nullptr,
                         const char** names = nullptr) {
  const bool with_adam = (mode == RUN_STEP);
  int launches = 0;
  int ne = 0;
  auto mark = [&](const char* name) {
    if (ev) {
      if (names && ne > 0) names[ne - 1] = name;
      cudaEventRecord(ev[ne++], s);
    }
  };
  dk::Bufs b = make_bufs(h);
  cudaError_t e = cudaMemsetAsync(h->counters.p, 0, 4 * sizeof(int), s);
  mark(nullptr);
  if (e == cudaSuccess && h->resample && h->rs_max > 0) {
    const int gx = (int)std::min<int64_t>((h->rs_max + 255) / 256, 64);
    dk::k_sample<<<dim3(gx, h->n_nets), 256, 0, s>>>(h->din, h->rs_seed, h->step_d.p, h->rs_off.p, h->rs_box.p,
                                                     h->res_pts.p);
    e = cudaGetLastError();
    ++launches;
    mark("sample");
  }
  b.no_reverse = (mode == RUN_LOSS) ? 1 : 0;
  // The residual-point jet items need no neighbour messages: without timing
  // events the exchange, face-jet and value items run on a side branch
  // (stream `side`, own stash) concurrently with them.  Timed runs keep
  // the kernels in sequence so that each gets its own interval.
  const bool fork = (ev == nullptr) && h->n_jet > 0 && (h->n_eval + h->n_val + h->n_jf) > 0;
  cudaStream_t s2 = fork ? h->side : s;
  if (e == cudaSuccess && fork) {
    e = cudaEventRecord(h->fork_ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, h->fork_ev, 0);
  }
  auto run_jet = [&]() {
    if (e == cudaSuccess && h->n_jet) {
      dk::Bufs bb = b;
      bb.counter = h->counters.p + 1;
      bb.stash_per_cta = h->ks.stash_train_jet;
      if (!stash_fits(h->stash, h->grid_jet, bb.stash_per_cta)) { e = cudaErrorInvalidValue; return; }
      e = launch_pinn(h->ks.train_jet_run, h->grid_jet, h->ks.smem_train_jet, h->shape, bb, h->items_jet.p,
                      h->n_items_d.p + 1, s, h->ks.threads_train_jet);
      ++launches;
      mark("train_jet");
    }
  };
  if (fork) run_jet();
  if (e == cudaSuccess && h->n_eval) {
    dk::Bufs bb = b;
    bb.counter = h->counters.p + 0;
    bb.no_reverse = 0;
    if (h->iface)   // the messages include the residual and first derivatives
      e = launch_pinn(h->ks.eval_jet, h->grid_eval, h->ks.smem_jet, h->shape, bb, h->items_eval.p, h->n_items_d.p + 0,
                      s2);
    else
      e = launch_pinn(h->ks.eval_val_run, h->grid_eval, h->ks.smem_val_run, h->shape, bb, h->items_eval.p,
                      h->n_items_d.p + 0, s2, h->ks.threads_val_run);
    ++launches;
    mark("exchange");
  }
  if (!fork) run_jet();
  if (e == cudaSuccess && h->n_jf) {   // face items with the interface jet terms (FP32 jet kernel)
    dk::Bufs bb = b;
    bb.counter = h->counters.p + 3;
    bb.stash = h->stash_side.p;   // sized for the side kernels, forked or in sequence
    bb.stash_per_cta = h->ks.stash_jet;
    e = stash_fits(h->stash_side, h->grid_jf, bb.stash_per_cta) ? cudaSuccess : cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = launch_pinn(h->ks.train_jet, h->grid_jf, h->ks.smem_jet, h->shape, bb, h->items_jf.p, h->n_items_d.p + 3, s2);
    ++launches;
    mark("train_face_jets");
  }
  if (e == cudaSuccess && h->n_val) {
    dk::Bufs bb = b;
    bb.counter = h->counters.p + 2;
    bb.stash = h->stash_side.p;
    bb.stash_per_cta = h->ks.stash_val_run;
    e = stash_fits(h->stash_side, h->grid_val, bb.stash_per_cta) ? cudaSuccess : cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = launch_pinn(h->ks.train_val_run, h->grid_val, h->ks.smem_val_run, h->shape, bb, h->items_val.p,
                    h->n_items_d.p + 2, s2, h->ks.threads_val_run);
    ++launches;
    mark("train_val");
  }
  if (fork) {   // joined even after an error, so that a capture ends cleanly
    cudaError_t ej = cudaEventRecord(h->join_ev, s2);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, h->join_ev, 0);
    if (e == cudaSuccess) e = ej;
  }
  const int nblk = (h->n_params + dk::NT - 1) / dk::NT;
  if (e == cudaSuccess && mode != RUN_LOSS) {
    dk::k_reduce_grad<<<dim3(nblk, h->n_nets), dk::NT, 0, s>>>(h->grad_part.p, h->slot_begin_d.p, h->grad.p,
                                                                h->norm_part.p, h->npp, h->n_params);
    e = cudaGetLastError();
    ++launches;
    mark("reduce_grad");
  }
  if (e == cudaSuccess && with_adam) {
    if (h->cfg.clip_norm > 0) {
      dk::k_clip_coef<<<h->n_nets, dk::NT, 0, s>>>(h->norm_part.p, nblk, (float)h->cfg.clip_norm, h->coef.p);
      ++launches;
      mark("clip");
    }
    const dk::AdamArgs ar = adam_args(h);
    dk::k_adam<<<dim3(nblk, h->n_nets), dk::NT, 0, s>>>(h->shape, ar, h->theta.p, h->thetaT.p, h->m.p, h->v.p,
                                                         h->grad.p, h->coef.p, h->step_d.p, h->n_params);
    e = cudaGetLastError();
    launches += 1;
    mark("adam");
  }
  if (e == cudaSuccess) {
    dk::k_loss_record<<<(h->n_nets + 3) / 4, 128, 0, s>>>(h->shape, h->loss_part.p, h->slot_begin_d.p,
                                                             h->nets_d.p, h->n_nets, h->loss_rec.p, h->err_d.p,
                                                             h->step_d.p, with_adam ? 1 : 0);
    e = cudaGetLastError();
    ++launches;
    mark("loss_record");
  }
  *n_launch = launches;
  return e;
}

int capture(dpinn* h, int mode, cudaGraphExec_t* out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaStream_t s = h->cap;
  CK(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int launches = 0;
  cudaError_t e = enqueue_step(h, mode, s, &launches);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(h, e, "capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  if (mode == RUN_STEP) h->launches = launches;
  return DPINN_OK;
}

// The kernels the step, the value items and the queries launch for an
// arithmetic (precision): the FP32 kernels, or at width 128 the tcgen05
// 3xTF32 ones, with their launch shapes and shared memory.
int select_kernels(dpinn* h, int precision) {
  if (precision == DPINN_PREC_TF32X3) {
    h->ks.train_jet_run = h->ks.train_jet_tc;
    h->ks.threads_train_jet = h->ks.threads_tc;
    h->ks.smem_train_jet = h->ks.smem_tc;
    h->ks.P_train_jet = h->ks.P_tc;
    h->ks.stash_train_jet = h->ks.stash_tc;
    h->ks.train_val_run = h->ks.train_val_tc;
    h->ks.eval_val_run = h->ks.eval_val_tc;
    h->ks.threads_val_run = h->ks.threads_tcv;
    h->ks.smem_val_run = h->ks.smem_tcv;
    h->ks.P_val_run = h->ks.P_tcv;
    h->ks.stash_val_run = h->ks.stash_tcv;
    h->ks.query_val_run = h->ks.query_val_tc;
    h->ks.query_jet_run = h->ks.query_jet_tc;
    h->ks.threads_qval = h->ks.threads_qjet = h->ks.threads_tcv;
    h->ks.P_qval = h->ks.P_tcv;
    h->ks.P_qjet = h->ks.P_tc;
    h->ks.smem_qval = h->ks.smem_tcv;
    h->ks.smem_qjet = h->ks.smem_tc;
  } else {
    // FP32: the default point tiles or, when selected and instantiated, the
    // alternate ones (dpinn_set_tiles)
    const bool aj = h->tile_jet != 0 && h->ks.train_jet_alt;
    const bool av = h->tile_val != 0 && h->ks.train_val_alt;
    h->ks.train_jet_run = aj ? h->ks.train_jet_alt : h->ks.train_jet;
    h->ks.threads_train_jet = dk::NT;
    h->ks.smem_train_jet = aj ? h->ks.smem_jet_alt : h->ks.smem_jet;
    h->ks.P_train_jet = aj ? h->ks.P_jet_alt : h->ks.P_jet;
    h->ks.stash_train_jet = aj ? h->ks.stash_jet_alt : h->ks.stash_jet;
    h->ks.train_val_run = av ? h->ks.train_val_alt : h->ks.train_val;
    h->ks.eval_val_run = av ? h->ks.eval_val_alt : h->ks.eval_val;
    h->ks.threads_val_run = dk::NT;
    h->ks.smem_val_run = av ? h->ks.smem_val_alt : h->ks.smem_val;
    h->ks.P_val_run = av ? h->ks.P_val_alt : h->ks.P_val;
    h->ks.stash_val_run = av ? h->ks.stash_val_alt : h->ks.stash_val;
    h->ks.query_val_run = h->ks.query_val;
    h->ks.query_jet_run = h->ks.query_jet;
    h->ks.threads_qval = h->ks.threads_qjet = dk::NT;
    h->ks.P_qval = h->ks.P_val;
    h->ks.P_qjet = h->ks.P_jet;
    h->ks.smem_qval = h->ks.smem_val;
    h->ks.smem_qjet = h->ks.smem_jet;
  }
  if (h->dev >= 0) {   // after creation: the chosen kernels' shared-memory limits
    if (h->ks.train_val_run != h->ks.train_val) {
      CK(h, cudaFuncSetAttribute(h->ks.query_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h->ks.smem_qval));
      CK(h, cudaFuncSetAttribute(h->ks.query_jet_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h->ks.smem_qjet));
      CK(h, cudaFuncSetAttribute(h->ks.train_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h->ks.smem_val_run));
      CK(h, cudaFuncSetAttribute(h->ks.eval_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h->ks.smem_val_run));
    }
    if (h->ks.train_jet_run != h->ks.train_jet)
      CK(h, cudaFuncSetAttribute(h->ks.train_jet_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h->ks.smem_train_jet));
  }
  h->cfg.precision = precision;
  return DPINN_OK;
}

int build_plan(dpinn* h) {
  h->plan_ok = false;
  if (!(h->have[0] && h->have[1] && (h->have[2] || h->n_faces == 0)))
    return DPINN_OK;   // built when every point set is present
  if (!h->have[2]) h->face_counts.assign(h->n_faces, 0);
  const int nn = h->n_nets;
  // Interfaces: the geometric faces (shared points, both sides train and
  // both evaluate) or, with volumetric ghost layers, directed segments (the
  // own net trains, the owner of the points evaluates).
  const bool directed = h->ghost_mode;
  std::vector<std::array<int, 3>> ifc;
  if (directed) ifc = h->seg;
  else
    for (auto& f : h->faces) ifc.push_back({f[0], f[1], (h->unst && f[2] == h->ds) ? 1 : 0});
  const std::vector<int64_t>& ifc_counts = directed ? h->seg_counts : h->face_counts;
  const int nf = (int)ifc.size();
  std::vector<std::vector<std::pair<int, int>>> trains(nn);   // (interface, side) per net
  for (int f = 0; f < nf; ++f) {
    trains[ifc[f][0]].push_back({f, 0});
    if (!directed) trains[ifc[f][1]].push_back({f, 1});
  }
  std::vector<int64_t> res_off(nn + 1, 0), obs_off(nn + 1, 0), face_off(nf + 1, 0);
  for (int k = 0; k < nn; ++k) res_off[k + 1] = res_off[k] + h->res_counts[k];
  for (int k = 0; k < nn; ++k) obs_off[k + 1] = obs_off[k] + h->obs_counts[k];
  for (int f = 0; f < nf; ++f) face_off[f + 1] = face_off[f] + ifc_counts[f];
  const int64_t n_face_pts = face_off[nf];

  // chunk sizes: enough items for several waves, multiples of the tile
  // (or the schedule set with dpinn_set_schedule)
  auto pick_chunk = [&](int64_t total, int P, int tiles) {
    if (tiles > 0) return (int64_t)tiles * P;
    const int64_t target = std::max<int64_t>(1, total / (8LL * h->n_sms));
    int64_t c = ((target + P - 1) / P) * P;
    return std::min<int64_t>(std::max<int64_t>(c, P), 64LL * P);
  };
  int64_t cj = pick_chunk(res_off[nn], h->ks.P_train_jet, h->sched_jet);
  int64_t cv = pick_chunk(obs_off[nn] + 2 * n_face_pts, h->ks.P_val_run, h->sched_val);
  // Every training item owns one gradient partial of npp floats: enlarge the
  // chunks until the partials fit the memory budget (at least one item per
  // net and point set remains), so the number of points per step is not
  // bounded by this memory.
  {
    auto n_slots = [&](int64_t a, int64_t b) {
      int64_t n = 0;
      for (int k = 0; k < nn; ++k) n += (h->res_counts[k] + a - 1) / a + (h->obs_counts[k] + b - 1) / b;
      for (int f = 0; f < nf; ++f) n += (directed ? 1 : 2) * ((ifc_counts[f] + b - 1) / b);
      return n;
    };
    const int64_t max_slots = std::max<int64_t>(1, h->part_budget / ((int64_t)h->npp * 4));
    const int64_t PJ = h->ks.P_train_jet, PV = h->ks.P_val_run;
    auto up = [](int64_t x, int64_t p) { return ((x + p - 1) / p) * p; };
    const int64_t cap_j = up(std::max<int64_t>(res_off[nn], 1), PJ);
    const int64_t cap_v = up(std::max<int64_t>(obs_off[nn] + n_face_pts, 1), PV);
    // chunks only grow and stop at the caps, so the loop ends
    while (n_slots(cj, cv) > max_slots) {
      const int64_t nj = std::max(cj, std::min(up(cj * 2, PJ), cap_j));
      const int64_t nv = std::max(cv, std::min(up(cv * 2, PV), cap_v));
      if (nj == cj && nv == cv) break;
      cj = nj;
      cv = nv;
    }
  }

  std::vector<dk::Item> ij, iv, ie, ijf;
  std::vector<int> slot_begin(nn + 1, 0);
  std::vector<dk::NetInfo> ni(nn);
  int slot = 0;
  for (int k = 0; k < nn; ++k) {
    slot_begin[k] = slot;
    chunks(res_off[k], h->res_counts[k], cj, [&](int64_t b, int64_t c) {
      ij.push_back({dk::K_PDE, k, (int)b, (int)c, slot++, 0, 0, 0});
    });
    chunks(obs_off[k], h->obs_counts[k], cv, [&](int64_t b, int64_t c) {
      iv.push_back({dk::K_OBS, k, (int)b, (int)c, slot++, 0, 0, 0});
    });
    int64_t ngh = 0;
    for (auto& fs : trains[k]) {
      const int f = fs.first, side = fs.second;
      ngh += ifc_counts[f];
      chunks(face_off[f], ifc_counts[f], cv, [&](int64_t b, int64_t c) {
        (h->iface ? ijf : iv).push_back({dk::K_FACE, k, (int)b, (int)c, slot++, f, side, 0});
      });
    }
    dk::NetInfo& n = ni[k];
    std::memset(&n, 0, sizeof(n));
    for (int q = 0; q < 4; ++q) {
      if (q < h->din) {
        n.center[q] = (float)(0.5 * (h->blo[k][q] + h->bhi[k][q]));
        n.scale[q] = (float)(2.0 / (h->bhi[k][q] - h->blo[k][q]));
      }
    }
    n.inv_npde = h->res_counts[k] ? (float)(1.0 / (double)h->res_counts[k]) : 0.f;
    n.inv_nobs = h->obs_counts[k] ? (float)(1.0 / (double)h->obs_counts[k]) : 0.f;
    n.inv_ngh = ngh ? (float)(1.0 / (double)ngh) : 0.f;
    n.master = h->master[k];
    n.lam_space = h->master[k] ? 0.f : (float)h->cfg.lambda_gh_p_space;
  }
  slot_begin[nn] = slot;
  h->n_slots = slot;
  for (int f = 0; f < nf; ++f)
    for (int side = directed ? 1 : 0; side < 2; ++side) {
      const int k = ifc[f][side];
      chunks(face_off[f], ifc_counts[f], cv, [&](int64_t b, int64_t c) {
        ie.push_back({dk::K_EVAL, k, (int)b, (int)c, 0, f, side, 0});
        if (h->master[k]) ie.push_back({dk::K_EVAL_ANC, k, (int)b, (int)c, 0, f, side, 0});
      });
    }
  {
    std::vector<int> fi((size_t)std::max(nf, 1) * 3, 0);
    for (int f = 0; f < nf; ++f)
      for (int q = 0; q < 3; ++q) fi[(size_t)f * 3 + q] = ifc[f][q];
    CK(h, h->face_info_d.ensure(fi.size()));
    CK(h, cudaMemcpy(h->face_info_d.p, fi.data(), fi.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  // longest chunks first (the scheduler hands items out in this order)
  auto by_count = [](const dk::Item& a, const dk::Item& b) { return a.count > b.count; };
  if (h->sched_order == 0) {
    std::stable_sort(ij.begin(), ij.end(), by_count);
    std::stable_sort(iv.begin(), iv.end(), by_count);
    std::stable_sort(ie.begin(), ie.end(), by_count);
  }
  h->n_jet = (int)ij.size();
  h->n_val = (int)iv.size();
  h->n_eval = (int)ie.size();
  h->n_jf = (int)ijf.size();

  const int occ_j = occupancy(h->ks.train_jet_run, h->ks.smem_train_jet, h->ks.threads_train_jet);
  const int occ_v = occupancy(h->ks.train_val_run, h->ks.smem_val_run, h->ks.threads_val_run);
  h->grid_jet = (int)std::min<int64_t>(h->n_jet, (int64_t)h->n_sms * occ_j);
  h->grid_val = (int)std::min<int64_t>(h->n_val, (int64_t)h->n_sms * occ_v);
  const int occ_e = h->iface ? occupancy(h->ks.eval_jet, h->ks.smem_jet)
                             : occupancy(h->ks.eval_val_run, h->ks.smem_val_run, h->ks.threads_val_run);
  h->grid_eval = (int)std::min<int64_t>(h->n_eval, (int64_t)h->n_sms * occ_e);
  const int occ_f = occupancy(h->ks.train_jet, h->ks.smem_jet);
  h->grid_jf = (int)std::min<int64_t>(h->n_jf, (int64_t)h->n_sms * occ_f);

  CK(h, h->items_jet.ensure(ij.size()));
  CK(h, h->items_val.ensure(iv.size()));
  CK(h, h->items_eval.ensure(ie.size()));
  CK(h, h->items_jf.ensure(ijf.size()));
  if (!ijf.empty())
    CK(h, cudaMemcpy(h->items_jf.p, ijf.data(), ijf.size() * sizeof(dk::Item), cudaMemcpyHostToDevice));
  if (!ij.empty()) CK(h, cudaMemcpy(h->items_jet.p, ij.data(), ij.size() * sizeof(dk::Item), cudaMemcpyHostToDevice));
  if (!iv.empty()) CK(h, cudaMemcpy(h->items_val.p, iv.data(), iv.size() * sizeof(dk::Item), cudaMemcpyHostToDevice));
  if (!ie.empty()) CK(h, cudaMemcpy(h->items_eval.p, ie.data(), ie.size() * sizeof(dk::Item), cudaMemcpyHostToDevice));
  int nitems[4] = {h->n_eval, h->n_jet, h->n_val, h->n_jf};
  CK(h, cudaMemcpy(h->n_items_d.p, nitems, sizeof(nitems), cudaMemcpyHostToDevice));
  CK(h, h->slot_begin_d.ensure(nn + 1));
  CK(h, cudaMemcpy(h->slot_begin_d.p, slot_begin.data(), (nn + 1) * sizeof(int), cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(h->nets_d.p, ni.data(), nn * sizeof(dk::NetInfo), cudaMemcpyHostToDevice));
  CK(h, h->grad_part.ensure((size_t)std::max(slot, 1) * h->npp));
  CK(h, h->loss_part.ensure((size_t)std::max(slot, 1) * dk::LP));
  CK(h, cudaMemset(h->loss_part.p, 0, (size_t)std::max(slot, 1) * dk::LP * sizeof(double)));
  const size_t st = (size_t)h->grid_jet * h->ks.stash_train_jet;
  const size_t st_side = std::max((size_t)h->grid_val * h->ks.stash_val_run, (size_t)h->grid_jf * h->ks.stash_jet);
  CK(h, h->stash.ensure(std::max<size_t>(st, 4)));
  CK(h, h->stash_side.ensure(std::max<size_t>(st_side, 4)));
  CK(h, h->nbr_val.ensure((size_t)std::max<int64_t>(n_face_pts, 1) * 2 * h->dout));
  CK(h, h->nbr_anc.ensure((size_t)std::max<int64_t>(n_face_pts, 1) * 2));
  if (h->iface) {
    CK(h, h->nbr_res.ensure((size_t)std::max<int64_t>(n_face_pts, 1) * 2 * (h->ds + 1)));
    CK(h, h->nbr_grd.ensure((size_t)std::max<int64_t>(n_face_pts, 1) * 2 * h->dout * h->din));
  }
  CK(h, cudaMemset(h->nbr_anc.p, 0, (size_t)std::max<int64_t>(n_face_pts, 1) * 2 * sizeof(float)));
  int rc = capture(h, RUN_STEP, &h->g_step);
  if (rc) return rc;
  rc = capture(h, RUN_GRAD, &h->g_grad);
  if (rc) return rc;
  rc = capture(h, RUN_LOSS, &h->g_loss);
  if (rc) return rc;
  h->plan_ok = true;
  return DPINN_OK;
}

int copy_state_in(dpinn* h, float* dst, const float* src) {
  CK(h, cudaMemcpy2D(dst, (size_t)h->npp * 4, src, (size_t)h->n_params * 4, (size_t)h->n_params * 4, h->n_nets,
                     cudaMemcpyDefault));
  return DPINN_OK;
}

int copy_state_out(dpinn* h, float* dst, const float* src) {
  CK(h, cudaMemcpy2D(dst, (size_t)h->n_params * 4, src, (size_t)h->npp * 4, (size_t)h->n_params * 4, h->n_nets,
                     cudaMemcpyDefault));
  return DPINN_OK;
}

int refresh_transpose(dpinn* h) {
  if (h->L < 2) return DPINN_OK;
  const int nblk = (h->nTp + dk::NT - 1) / dk::NT;
  dk::k_transpose<<<dim3(nblk, h->n_nets), dk::NT>>>(h->shape, h->theta.p, h->thetaT.p);
  CK(h, cudaGetLastError());
  CK(h, cudaDeviceSynchronize());
  return DPINN_OK;
}

int check_errors(dpinn* h) {
  int e[3] = {0, 0, 0};
  CK(h, cudaMemcpy(e, h->err_d.p, sizeof(e), cudaMemcpyDeviceToHost));
  if (e[dk::ERR_TIMEOUT]) return fail(h, DPINN_ERR_TIMEOUT, "a device wait gave up (bulk copy never completed)");
  if (e[dk::ERR_NONFINITE]) {
    CK(h, cudaMemset(h->err_d.p + dk::ERR_NONFINITE, 0, sizeof(int)));
    return fail(h, DPINN_ERR_NONFINITE, "non-finite loss");
  }
  return DPINN_OK;
}

// Device scratch of one query launch sequence (routing and work items).
struct QueryScratch {
  int *net_of, *perm, *counts, *offsets, *cursor, *nitems;
  dk::Item* items;
  int* err;          // error words the route and query kernels report to
  size_t items_cap;  // capacity of `items`
};

// Query modes: values, values + Navier-Stokes residuals, raw output jets.
enum { Q_VALUES = 0, Q_RESIDUAL = 1, Q_JETS = 2 };

// Points per work item of a query in `mode` (four tiles of its kernel).
int64_t query_chunk(const dpinn* h, int mode) { return 4 * (int64_t)(mode == Q_VALUES ? h->ks.P_qval : h->ks.P_qjet); }

// Upper bound of the work items of an n-point query: one per started chunk
// of every net's segment.
size_t query_max_items(const dpinn* h, int64_t n, int mode) {
  return (size_t)(n / query_chunk(h, mode)) + h->n_nets + 1;
}

// Route n points to their nets, order them by net, build the work items and
// launch the grouped query kernel, all on stream s.
int enqueue_query(dpinn* h, const QueryScratch& q, const float* pts, int64_t n, int mode, float* out,
                  cudaStream_t s) {
  const int chunk = (int)query_chunk(h, mode);
  const size_t max_items = query_max_items(h, n, mode);
  if (max_items > q.items_cap) return fail(h, DPINN_ERR_STATE, "query work-item scratch too small");
  dk::Route rt{};
  for (int a = 0; a < h->din; ++a) {
    rt.lo[a] = (float)h->cfg.lo[a];
    rt.hi[a] = (float)h->cfg.hi[a];
    rt.inv_h[a] = (float)((double)h->cfg.splits[a] / (h->cfg.hi[a] - h->cfg.lo[a]));
    rt.splits[a] = h->cfg.splits[a];
    rt.stride[a] = h->stride[a];
  }
  rt.din = h->din;
  rt.n_nets = h->n_nets;
  CK(h, cudaMemsetAsync(q.counts, 0, h->n_nets * sizeof(int), s));
  CK(h, cudaMemsetAsync(q.nitems, 0, 2 * sizeof(int), s));
  const int nb = (int)((n + 255) / 256);
  dk::k_route<<<nb, 256, 0, s>>>(rt, pts, n, q.net_of, q.counts, q.err);
  dk::k_route_plan<<<1, 32, 0, s>>>(q.counts, h->n_nets, chunk, q.offsets, q.cursor, q.items, q.nitems);
  dk::k_route_scatter<<<nb, 256, 0, s>>>(q.net_of, n, q.cursor, q.perm);
  CK(h, cudaGetLastError());
  dk::Bufs b = make_bufs(h);
  b.counter = q.nitems + 1;
  b.err = q.err;
  b.q_pts = pts;
  b.q_perm = q.perm;
  b.q_out = out;
  b.q_jets = mode == Q_JETS ? 1 : 0;
  b.q_w = mode == Q_JETS ? h->dout * (h->din + 2) : h->dout + (mode == Q_RESIDUAL ? h->ds + 1 : 0);
  const bool jet = mode != Q_VALUES;
  const void* fn = jet ? h->ks.query_jet_run : h->ks.query_val_run;
  const size_t smem = jet ? h->ks.smem_qjet : h->ks.smem_qval;
  const int threads = jet ? h->ks.threads_qjet : h->ks.threads_qval;
  // One CTA per work item rather than a persistent grid: CTAs retire as their
  // items finish, so the block scheduler can interleave the kernels of other
  // (higher-priority) streams with a large query.
  const int grid = (int)std::min<size_t>(max_items, (size_t)1 << 30);
  CK(h, launch_pinn(fn, grid, smem, h->shape, b, q.items, q.nitems, s, threads));
  return DPINN_OK;
}

// dpinn_query / dpinn_query_jets: routing scratch owned by the handle, grown
// to the largest request so far.
int handle_query(dpinn* h, const float* pts, int64_t n, int mode, float* out, cudaStream_t s) {
  if (n < 0 || n > ((int64_t)1 << 30)) return fail(h, DPINN_ERR_INVALID_ARG, "bad point count");
  if (n == 0) return DPINN_OK;
  if (!pts || !out) return fail(h, DPINN_ERR_INVALID_ARG, "null pointer");
  const size_t max_items = query_max_items(h, n, mode);
  CK(h, h->q_net.ensure(n));
  CK(h, h->q_perm.ensure(n));
  CK(h, h->q_counts.ensure(h->n_nets));
  CK(h, h->q_off.ensure(h->n_nets));
  CK(h, h->q_cursor.ensure(h->n_nets));
  CK(h, h->q_nitems.ensure(2));
  CK(h, h->q_items.ensure(max_items));
  QueryScratch qs{h->q_net.p, h->q_perm.p, h->q_counts.p, h->q_off.p, h->q_cursor.p, h->q_nitems.p,
                  h->q_items.p, h->err_d.p, max_items};
  return enqueue_query(h, qs, pts, n, mode, out, s);
}

}  // namespace

// Query context: its own scratch (sized once at creation) and error words, so
// that queries on several streams can be in flight together.
// All of a context's device scratch is one allocation (its parts 256-byte
// aligned), so that a caller budgeting device memory (the serving loop) pays
// the allocator's rounding once per context.
struct dpinn_qctx {
  dpinn* h = nullptr;
  int64_t cap = 0;
  size_t items_cap = 0;
  DevBuf<unsigned char> mem;
  int *net_of = nullptr, *perm = nullptr, *counts = nullptr, *offsets = nullptr, *cursor = nullptr,
      *nitems = nullptr, *err = nullptr;
  dk::Item* items = nullptr;
  ~dpinn_qctx() { mem.free_(); }
};

// =================================================================== ABI ===
extern "C" {

int dpinn_config_default(dpinn_config* c) {
  if (!c) return DPINN_ERR_INVALID_ARG;
  std::memset(c, 0, sizeof(*c));
  c->d_space = 2;
  for (int a = 0; a < 4; ++a) { c->lo[a] = 0.0; c->hi[a] = 1.0; c->splits[a] = 1; }
  c->depth = 4;
  c->width = 32;
  c->nu = 0.01;
  c->lambda_obs = c->lambda_pde = c->lambda_gh_u = c->lambda_gh_p_space = c->lambda_gh_p_time = 1.0;
  c->comp_w[0] = c->comp_w[1] = c->comp_w[2] = 1.0;
  c->lr = 1e-3; c->beta1 = 0.9; c->beta2 = 0.999; c->eps = 1e-8;
  c->lr_decay_factor = 1.0;
  c->lr_decay_interval = 0;
  c->comm_interval = 1;
  c->lambda_gh_r = c->lambda_gh_c1 = 0.0;
  return DPINN_OK;
}

const char* dpinn_last_error(dpinn_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int dpinn_create(const dpinn_config* cfg, dpinn_t** out) {
  if (!cfg || !out) return fail(nullptr, DPINN_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const dpinn_config& c = *cfg;
  if (c.d_space != 2 && c.d_space != 3) return fail(nullptr, DPINN_ERR_INVALID_ARG, "d_space must be 2 or 3");
  if (c.unsteady != 0 && c.unsteady != 1) return fail(nullptr, DPINN_ERR_INVALID_ARG, "unsteady must be 0 or 1");
  if (c.width != 32 && c.width != 64 && !(c.width >= 128 && c.width <= 224))
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "width must be 32, 64 or in [128, 224]");
  if (c.depth < 1 || c.depth > dk::MAXL) return fail(nullptr, DPINN_ERR_INVALID_ARG, "depth must be in [1, 16]");
  if (c.activation != DPINN_ACT_TANH && c.activation != DPINN_ACT_SIN)
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "activation must be tanh or sin");
  if (c.precision != DPINN_PREC_FP32 && c.precision != DPINN_PREC_TF32X3)
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "precision must be FP32 or TF32x3");
  if (c.precision == DPINN_PREC_TF32X3 && c.width != 128)
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "TF32x3 tensor-core kernels need width 128");
  if (!(c.nu >= 0)) return fail(nullptr, DPINN_ERR_INVALID_ARG, "nu must be >= 0");
  if (c.comm_interval < 1) return fail(nullptr, DPINN_ERR_INVALID_ARG, "comm_interval must be >= 1");
  if (!(c.lambda_gh_r >= 0.0) || !(c.lambda_gh_c1 >= 0.0))
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "interface weights must be >= 0");
  if (!(c.beta1 >= 0 && c.beta1 < 1) || !(c.beta2 >= 0 && c.beta2 < 1))
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "Adam betas must be in [0, 1)");
  if (c.lr_decay_interval < 0 || !(c.lr_decay_factor > 0))
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "bad learning-rate decay");
  const int din = c.d_space + c.unsteady;
  int64_t nn = 1;
  for (int a = 0; a < din; ++a) {
    if (c.splits[a] < 1) return fail(nullptr, DPINN_ERR_INVALID_ARG, "splits must be >= 1");
    if (!(c.hi[a] > c.lo[a])) return fail(nullptr, DPINN_ERR_INVALID_ARG, "hi must exceed lo");
    nn *= c.splits[a];
  }
  if (nn > 65535) return fail(nullptr, DPINN_ERR_INVALID_ARG, "too many nets");
  for (int a = 0; a < c.d_space; ++a)
    if (cell_fp32(c, a, (float)c.anchor_x[a]) < 0) return fail(nullptr, DPINN_ERR_INVALID_ARG, "anchor outside the domain");

  std::unique_ptr<dpinn> h(new dpinn());
  h->cfg = c;
  h->ds = c.d_space; h->unst = c.unsteady; h->din = din; h->dout = c.d_space + 1;
  h->W = c.width; h->L = c.depth;
  h->n_nets = (int)nn;
  if (!pick_kernels(h->W, h->ds, h->unst, h->L, c.activation, &h->ks))
    return fail(nullptr, DPINN_ERR_INVALID_ARG, "unsupported shape");
  h->dev = -1;
  select_kernels(h.get(), c.precision);
  // decomposition
  int s = 1;
  for (int a = 0; a < din; ++a) { h->stride.push_back(s); s *= c.splits[a]; }
  for (int k = 0; k < h->n_nets; ++k) {
    std::array<int, 4> ce{0, 0, 0, 0};
    std::array<double, 4> lo{0, 0, 0, 0}, hi{0, 0, 0, 0};
    int r = k;
    for (int a = 0; a < din; ++a) {
      ce[a] = r % c.splits[a];
      r /= c.splits[a];
      const double hh = (c.hi[a] - c.lo[a]) / c.splits[a];
      lo[a] = c.lo[a] + ce[a] * hh;
      hi[a] = c.lo[a] + (ce[a] + 1) * hh;
    }
    h->cell.push_back(ce); h->blo.push_back(lo); h->bhi.push_back(hi);
  }
  int acell[3] = {0, 0, 0};
  for (int a = 0; a < h->ds; ++a) acell[a] = cell_fp32(c, a, (float)c.anchor_x[a]);
  for (int k = 0; k < h->n_nets; ++k) {
    bool mm = true;
    for (int a = 0; a < h->ds; ++a) mm = mm && h->cell[k][a] == acell[a];
    h->master.push_back(mm ? 1 : 0);
  }
  h->net_faces.resize(h->n_nets);
  for (int a = 0; a < din; ++a)
    for (int k = 0; k < h->n_nets; ++k)
      if (h->cell[k][a] < c.splits[a] - 1) {
        const int f = (int)h->faces.size();
        h->faces.push_back({k, k + h->stride[a], a});
        h->net_faces[k].push_back(f);
        h->net_faces[k + h->stride[a]].push_back(f);
      }
  h->n_faces = (int)h->faces.size();
  // parameter layout
  dk::Shape& sh = h->shape;
  std::memset(&sh, 0, sizeof(sh));
  sh.ds = h->ds; sh.unst = h->unst; sh.din = din; sh.dout = h->dout; sh.W = h->W; sh.L = h->L;
  int off = 0;
  for (int l = 0; l <= h->L; ++l) {
    const int o = (l == h->L) ? h->dout : h->W;
    const int i = (l == 0) ? din : h->W;
    sh.woff[l] = off; off += o * i;
    sh.boff[l] = off; off += o;
  }
  h->n_params = off;
  h->npp = ((off + 63) / 64) * 64;
  // the tensor-core kernels move each hidden-layer weight-gradient tile of a
  // slot with one bulk operation, which needs a 16-byte aligned address (true
  // for W = 128: every woff[l], l >= 1, is a multiple of 128 floats)
  if (c.precision == DPINN_PREC_TF32X3)
    for (int l = 1; l < h->L; ++l)
      if (sh.woff[l] % 4 != 0) return fail(nullptr, DPINN_ERR_INVALID_ARG, "weight-gradient tile not 16-byte aligned");
  // widths 129-224 run the streamed-weight kernels (padded to 160 or 224),
  // whose hidden weights are kept in their own lane-blocked layout
  sh.twp = (h->W > 128) ? (h->W <= 160 ? 160 : 224) : 0;
  h->nTp = std::max(1, sh.twp ? (h->L - 1) * 2 * h->W * sh.twp : (h->L - 1) * h->W * h->W);
  sh.npp = h->npp; sh.nTp = h->nTp;
  sh.act = (c.activation == DPINN_ACT_SIN) ? dk::ACT_SIN : dk::ACT_TANH;
  sh.nu = (float)c.nu; sh.p_ref = (float)c.p_ref;
  for (int a = 0; a < 3; ++a) { sh.anchor[a] = (float)c.anchor_x[a]; sh.comp_w[a] = (float)c.comp_w[a]; }
  sh.lam_obs = (float)c.lambda_obs; sh.lam_pde = (float)c.lambda_pde; sh.lam_gh_u = (float)c.lambda_gh_u;
  sh.lam_time = (float)c.lambda_gh_p_time;
  sh.lam_gh_r = (float)c.lambda_gh_r;
  sh.lam_gh_c1 = (float)c.lambda_gh_c1;
  h->iface = (c.lambda_gh_r != 0.0 || c.lambda_gh_c1 != 0.0);

  dpinn* hp = h.get();
  CK(hp, cudaSetDevice(c.device));
  h->dev = c.device;
  CK(hp, cudaDeviceGetAttribute(&h->n_sms, cudaDevAttrMultiProcessorCount, c.device));
  for (const void* fn : {h->ks.train_jet, h->ks.query_jet})
    CK(hp, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem_jet));
  CK(hp, cudaFuncSetAttribute(h->ks.eval_jet, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem_jet));
  if (h->ks.train_val_run != h->ks.train_val) {
    CK(hp, cudaFuncSetAttribute(h->ks.query_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)h->ks.smem_qval));
    CK(hp, cudaFuncSetAttribute(h->ks.query_jet_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)h->ks.smem_qjet));
    CK(hp, cudaFuncSetAttribute(h->ks.train_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)h->ks.smem_val_run));
    CK(hp, cudaFuncSetAttribute(h->ks.eval_val_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)h->ks.smem_val_run));
  }
  if (h->ks.train_jet_run != h->ks.train_jet)
    CK(hp, cudaFuncSetAttribute(h->ks.train_jet_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)h->ks.smem_train_jet));
  for (const void* fn : {h->ks.train_val, h->ks.eval_val, h->ks.query_val})
    CK(hp, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->ks.smem_val));
  const size_t NP = (size_t)h->n_nets * h->npp;
  CK(hp, h->theta.ensure(NP)); CK(hp, h->m.ensure(NP)); CK(hp, h->v.ensure(NP)); CK(hp, h->grad.ensure(NP));
  CK(hp, h->thetaT.ensure((size_t)h->n_nets * h->nTp));
  const int nblk = (h->n_params + dk::NT - 1) / dk::NT;
  CK(hp, h->norm_part.ensure((size_t)h->n_nets * nblk));
  CK(hp, h->coef.ensure(h->n_nets));
  CK(hp, h->step_d.ensure(1));
  CK(hp, h->nets_d.ensure(h->n_nets));
  CK(hp, h->face_info_d.ensure((size_t)std::max(h->n_faces, 1) * 3));
  CK(hp, h->err_d.ensure(4)); CK(hp, h->counters.ensure(4)); CK(hp, h->n_items_d.ensure(4));
  CK(hp, h->loss_rec.ensure((size_t)h->n_nets * 8));
  CK(hp, h->iota_d.ensure(h->n_nets + 1));
  CK(hp, cudaMallocHost(&h->loss_host, (size_t)h->n_nets * 8 * sizeof(float)));
  CK(hp, cudaMemset(h->theta.p, 0, NP * 4)); CK(hp, cudaMemset(h->m.p, 0, NP * 4));
  CK(hp, cudaMemset(h->v.p, 0, NP * 4)); CK(hp, cudaMemset(h->grad.p, 0, NP * 4));
  CK(hp, cudaMemset(h->step_d.p, 0, sizeof(long long)));
  CK(hp, cudaMemset(h->err_d.p, 0, 4 * sizeof(int)));
  CK(hp, cudaMemset(h->loss_rec.p, 0, (size_t)h->n_nets * 8 * sizeof(float)));
  CK(hp, cudaMemset(h->coef.p, 0, (size_t)h->n_nets * sizeof(float)));
  std::vector<int> fi((size_t)std::max(h->n_faces, 1) * 3, 0);
  for (int f = 0; f < h->n_faces; ++f) {
    fi[f * 3] = h->faces[f][0];
    fi[f * 3 + 1] = h->faces[f][1];
    fi[f * 3 + 2] = (h->unst && h->faces[f][2] == h->ds) ? 1 : 0;
  }
  CK(hp, cudaMemcpy(h->face_info_d.p, fi.data(), fi.size() * sizeof(int), cudaMemcpyHostToDevice));
  std::vector<int> iota(h->n_nets + 1);
  for (int k = 0; k <= h->n_nets; ++k) iota[k] = k;
  CK(hp, cudaMemcpy(h->iota_d.p, iota.data(), iota.size() * sizeof(int), cudaMemcpyHostToDevice));
  // empty per-net info until points arrive
  std::vector<dk::NetInfo> ni(h->n_nets);
  for (int k = 0; k < h->n_nets; ++k) {
    std::memset(&ni[k], 0, sizeof(dk::NetInfo));
    for (int q = 0; q < din; ++q) {
      ni[k].center[q] = (float)(0.5 * (h->blo[k][q] + h->bhi[k][q]));
      ni[k].scale[q] = (float)(2.0 / (h->bhi[k][q] - h->blo[k][q]));
    }
    ni[k].master = h->master[k];
    ni[k].lam_space = h->master[k] ? 0.f : (float)c.lambda_gh_p_space;
  }
  CK(hp, cudaMemcpy(h->nets_d.p, ni.data(), ni.size() * sizeof(dk::NetInfo), cudaMemcpyHostToDevice));
  dk::k_init<<<dim3(nblk, h->n_nets), dk::NT>>>(h->shape, (uint64_t)c.seed, h->theta.p, h->n_params);
  CK(hp, cudaGetLastError());
  int rc = refresh_transpose(hp);
  if (rc) { g_create_err = h->err; return rc; }
  CK(hp, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(hp, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CK(hp, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
  CK(hp, cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
  CK(hp, cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
  CK(hp, cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
  CK(hp, cudaEventCreateWithFlags(&h->stage_ready, cudaEventDisableTiming));
  CK(hp, cudaEventCreateWithFlags(&h->stage_free, cudaEventDisableTiming));
  CK(hp, cudaEventRecord(h->stage_free, h->copy_st));
  CK(hp, cudaDeviceSynchronize());
  *out = h.release();
  return DPINN_OK;
}

void dpinn_destroy(dpinn_t* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  cudaDeviceSynchronize();
  delete h;
}

int dpinn_get_layout(dpinn_t* h, dpinn_layout* o) {
  if (!h || !o) return DPINN_ERR_INVALID_ARG;
  o->n_nets = h->n_nets; o->n_faces = h->n_faces; o->d_in = h->din; o->d_out = h->dout;
  o->n_params = h->n_params;
  int nm = 0;
  for (int x : h->master) nm += x;
  o->n_masters = nm;
  return DPINN_OK;
}

int dpinn_net_info(dpinn_t* h, int net, int* is_master, double* lo4, double* hi4) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (net < 0 || net >= h->n_nets) return fail(h, DPINN_ERR_INVALID_ARG, "net out of range");
  if (is_master) *is_master = h->master[net];
  for (int q = 0; q < 4; ++q) {
    if (lo4) lo4[q] = h->blo[net][q];
    if (hi4) hi4[q] = h->bhi[net][q];
  }
  return DPINN_OK;
}

int dpinn_face_info(dpinn_t* h, int f, int* lo, int* hi, int* axis, int* is_time) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (f < 0 || f >= h->n_faces) return fail(h, DPINN_ERR_INVALID_ARG, "face out of range");
  if (lo) *lo = h->faces[f][0];
  if (hi) *hi = h->faces[f][1];
  if (axis) *axis = h->faces[f][2];
  if (is_time) *is_time = (h->unst && h->faces[f][2] == h->ds) ? 1 : 0;
  return DPINN_OK;
}

namespace {
// Volumetric ghost points: route every point of net A to the net B whose
// cell holds it (float32 rule), group A's points by B into directed
// segments (A, B, is_time), and upload them in segment order.
int set_ghost_points(dpinn* h, const float* pts, const int64_t* counts) {
  int64_t n = 0;
  for (int k = 0; k < h->n_nets; ++k) n += counts[k];
  std::vector<float> hp((size_t)n * h->din);
  if (n) CK(h, cudaMemcpy(hp.data(), pts, hp.size() * sizeof(float), cudaMemcpyDefault));
  std::vector<std::array<int, 3>> seg;
  std::vector<int64_t> seg_counts;
  std::vector<float> sorted;
  sorted.reserve(hp.size());
  int64_t off = 0;
  for (int A = 0; A < h->n_nets; ++A) {
    std::vector<std::pair<int, int64_t>> own;   // (owner, point index)
    for (int64_t i = off; i < off + counts[A]; ++i) {
      int B = 0;
      for (int a = 0; a < h->din; ++a) {
        const int c = cell_fp32(h->cfg, a, hp[(size_t)i * h->din + a]);
        if (c < 0) return fail(h, DPINN_ERR_INVALID_ARG, "ghost point outside the domain");
        B += c * h->stride[a];
      }
      if (B == A) return fail(h, DPINN_ERR_INVALID_ARG, "ghost point inside its own net's cell");
      own.push_back({B, i});
    }
    off += counts[A];
    std::stable_sort(own.begin(), own.end(),
                     [](const std::pair<int, int64_t>& x, const std::pair<int, int64_t>& y) { return x.first < y.first; });
    for (size_t j = 0; j < own.size(); ++j) {
      const int B = own[j].first;
      if (j == 0 || own[j - 1].first != B) {
        bool same_space = true;
        for (int a = 0; a < h->ds; ++a) same_space = same_space && h->cell[A][a] == h->cell[B][a];
        seg.push_back({A, B, (h->unst && same_space) ? 1 : 0});
        seg_counts.push_back(0);
      }
      seg_counts.back() += 1;
      for (int q = 0; q < h->din; ++q) sorted.push_back(hp[(size_t)own[j].second * h->din + q]);
    }
  }
  CK(h, cudaDeviceSynchronize());
  CK(h, h->face_pts.ensure((size_t)std::max<int64_t>(n, 1) * h->din));
  if (n) CK(h, cudaMemcpy(h->face_pts.p, sorted.data(), sorted.size() * sizeof(float), cudaMemcpyHostToDevice));
  h->seg = seg;
  h->seg_counts = seg_counts;
  h->ghost_mode = true;
  h->have[2] = true;
  return build_plan(h);
}
}  // namespace

int dpinn_set_points(dpinn_t* h, int kind, const float* pts, const float* vals, const int64_t* counts, int n_counts) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (kind < 0 || kind > 3) return fail(h, DPINN_ERR_INVALID_ARG, "bad point kind");
  if (kind == DPINN_POINTS_GHOST) {
    if (n_counts != h->n_nets || !counts) return fail(h, DPINN_ERR_INVALID_ARG, "counts length mismatch");
    int64_t n = 0;
    for (int i = 0; i < n_counts; ++i) {
      if (counts[i] < 0) return fail(h, DPINN_ERR_INVALID_ARG, "negative count");
      n += counts[i];
    }
    if (n > (int64_t)1 << 30) return fail(h, DPINN_ERR_INVALID_ARG, "too many points");
    if (n > 0 && !pts) return fail(h, DPINN_ERR_INVALID_ARG, "null points");
    CK(h, cudaSetDevice(h->dev));
    return set_ghost_points(h, pts, counts);
  }
  const int expect = kind == DPINN_POINTS_FACE ? h->n_faces : h->n_nets;
  if (n_counts != expect || (!counts && expect > 0)) return fail(h, DPINN_ERR_INVALID_ARG, "counts length mismatch");
  int64_t n = 0;
  for (int i = 0; i < n_counts; ++i) {
    if (counts[i] < 0) return fail(h, DPINN_ERR_INVALID_ARG, "negative count");
    n += counts[i];
  }
  if (n > (int64_t)1 << 30) return fail(h, DPINN_ERR_INVALID_ARG, "too many points");
  if (n > 0 && !pts) return fail(h, DPINN_ERR_INVALID_ARG, "null points");
  if (kind == DPINN_POINTS_OBS && n > 0 && !vals) return fail(h, DPINN_ERR_INVALID_ARG, "null observation values");
  CK(h, cudaSetDevice(h->dev));
  if (kind == DPINN_POINTS_RESIDUAL && h->stage_pending) {   // the new points replace a pending upload
    CK(h, cudaStreamSynchronize(h->copy_st));
    h->stage_pending = false;
  }
  std::vector<int64_t> cv(counts, counts + n_counts);
  std::vector<int64_t>* dst = kind == 0 ? &h->res_counts : (kind == 1 ? &h->obs_counts : &h->face_counts);
  // points delivered by the caller replace per-step resampling
  const bool was_sampling = (kind == DPINN_POINTS_RESIDUAL) && h->resample;
  if (was_sampling) h->resample = false;
  const bool same = h->have[kind] && *dst == cv && !was_sampling;
  DevBuf<float>* pb = kind == 0 ? &h->res_pts : (kind == 1 ? &h->obs_pts : &h->face_pts);
  if (!same) {
    // the captured graphs reference the old buffers: drop them first
    CK(h, cudaDeviceSynchronize());
  }
  CK(h, pb->ensure((size_t)std::max<int64_t>(n, 1) * h->din));
  if (n) CK(h, cudaMemcpy(pb->p, pts, (size_t)n * h->din * sizeof(float), cudaMemcpyDefault));
  if (kind == DPINN_POINTS_OBS) {
    CK(h, h->obs_vals.ensure((size_t)std::max<int64_t>(n, 1) * h->ds));
    if (n) CK(h, cudaMemcpy(h->obs_vals.p, vals, (size_t)n * h->ds * sizeof(float), cudaMemcpyDefault));
  }
  *dst = cv;
  h->have[kind] = true;
  if (kind == DPINN_POINTS_FACE && h->ghost_mode) {
    h->ghost_mode = false;
    return build_plan(h);
  }
  if (same && h->plan_ok) return DPINN_OK;
  return build_plan(h);
}

// A pending asynchronous upload enters res_pts on the launching stream just
// before the work that reads it.
static int apply_stage(dpinn* h, cudaStream_t s) {
  if (!h->stage_pending) return DPINN_OK;
  CK(h, cudaStreamWaitEvent(s, h->stage_ready, 0));
  CK(h, cudaMemcpyAsync(h->res_pts.p, h->res_stage.p, h->stage_bytes, cudaMemcpyDeviceToDevice, s));
  CK(h, cudaEventRecord(h->stage_free, s));
  h->stage_pending = false;
  return DPINN_OK;
}

int dpinn_set_points_async(dpinn_t* h, int kind, const float* pts, const int64_t* counts, int n_counts,
                           dpinn_stream_t stream) {
  (void)stream;
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (kind != DPINN_POINTS_RESIDUAL) return fail(h, DPINN_ERR_INVALID_ARG, "asynchronous upload of residual points only");
  if (n_counts != h->n_nets || !counts) return fail(h, DPINN_ERR_INVALID_ARG, "counts length mismatch");
  const bool same = h->have[0] && !h->resample &&
                    std::equal(counts, counts + n_counts, h->res_counts.begin(), h->res_counts.end());
  if (!same)   // a new layout needs a new plan: the synchronous path
    return dpinn_set_points(h, kind, pts, nullptr, counts, n_counts);
  int64_t n = 0;
  for (int i = 0; i < n_counts; ++i) n += counts[i];
  if (n == 0) return DPINN_OK;
  if (!pts) return fail(h, DPINN_ERR_INVALID_ARG, "null points");
  CK(h, cudaSetDevice(h->dev));
  const size_t bytes = (size_t)n * h->din * sizeof(float);
  if (h->stage_pending) return fail(h, DPINN_ERR_STATE, "an earlier asynchronous upload has not been consumed");
  if (h->res_stage.n < (size_t)n * h->din) {
    CK(h, cudaEventSynchronize(h->stage_free));
    CK(h, h->res_stage.ensure((size_t)n * h->din));
  }
  CK(h, cudaStreamWaitEvent(h->copy_st, h->stage_free, 0));   // the previous upload has been moved out
  CK(h, cudaMemcpyAsync(h->res_stage.p, pts, bytes, cudaMemcpyHostToDevice, h->copy_st));
  CK(h, cudaEventRecord(h->stage_ready, h->copy_st));
  h->stage_bytes = bytes;
  h->stage_pending = true;
  return DPINN_OK;
}

int dpinn_selftest_wait(dpinn_t* h) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaSetDevice(h->dev));
  DevBuf<int> e;
  CK(h, e.ensure(3));
  CK(h, cudaMemset(e.p, 0, 3 * sizeof(int)));
  dk::k_selftest_wait<<<1, 32>>>(e.p);
  CK(h, cudaGetLastError());
  CK(h, cudaDeviceSynchronize());
  int w[3] = {0, 0, 0};
  CK(h, cudaMemcpy(w, e.p, sizeof(w), cudaMemcpyDeviceToHost));
  e.free_();
  if (w[dk::ERR_TIMEOUT]) return fail(h, DPINN_ERR_TIMEOUT, "self-test: the bounded wait gave up as designed");
  return fail(h, DPINN_ERR_STATE, "self-test: a wait that nothing completes returned without a time-out");
}

int dpinn_selftest_sincos(int device, const float* x, long long n, float* out) {
  if (n < 0 || (n > 0 && (!x || !out))) return DPINN_ERR_INVALID_ARG;
  if (n == 0) return DPINN_OK;
  if (cudaSetDevice(device) != cudaSuccess) return DPINN_ERR_CUDA;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  dk::k_selftest_sincos<<<(unsigned)blocks, 256>>>(x, n, out);
  if (cudaGetLastError() != cudaSuccess) return DPINN_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? DPINN_OK : DPINN_ERR_CUDA;
}

int dpinn_set_resampling(dpinn_t* h, const int64_t* counts, int n_counts, uint64_t seed) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (!counts) {
    if (h->resample) {
      CK(h, cudaSetDevice(h->dev));
      CK(h, cudaDeviceSynchronize());
      h->resample = false;
      h->plan_ok = false;
      return build_plan(h);
    }
    return DPINN_OK;
  }
  if (n_counts != h->n_nets) return fail(h, DPINN_ERR_INVALID_ARG, "counts length mismatch");
  int64_t n = 0, mx = 0;
  for (int i = 0; i < n_counts; ++i) {
    if (counts[i] < 0) return fail(h, DPINN_ERR_INVALID_ARG, "negative count");
    n += counts[i];
    mx = std::max<int64_t>(mx, counts[i]);
  }
  if (n > (int64_t)1 << 30) return fail(h, DPINN_ERR_INVALID_ARG, "too many points");
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaDeviceSynchronize());   // the captured graphs reference the old buffers
  std::vector<long long> off(h->n_nets + 1, 0);
  std::vector<double> box((size_t)h->n_nets * 8, 0.0);
  for (int k = 0; k < h->n_nets; ++k) {
    off[k + 1] = off[k] + counts[k];
    for (int q = 0; q < h->din; ++q) {
      box[(size_t)k * 8 + q] = h->blo[k][q];
      box[(size_t)k * 8 + 4 + q] = h->bhi[k][q] - h->blo[k][q];
    }
  }
  CK(h, h->rs_off.ensure(off.size()));
  CK(h, cudaMemcpy(h->rs_off.p, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
  CK(h, h->rs_box.ensure(box.size()));
  CK(h, cudaMemcpy(h->rs_box.p, box.data(), box.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(h, h->res_pts.ensure((size_t)std::max<int64_t>(n, 1) * h->din));
  h->res_counts.assign(counts, counts + n_counts);
  h->have[0] = true;
  h->resample = true;
  h->rs_seed = seed;
  h->rs_max = mx;
  h->plan_ok = false;
  return build_plan(h);
}

int dpinn_get_points(dpinn_t* h, int kind, float* host_out) {
  if (!h || !host_out) return DPINN_ERR_INVALID_ARG;
  if (kind < 0 || kind > 2) return fail(h, DPINN_ERR_INVALID_ARG, "bad point kind");
  if (!h->have[kind]) return fail(h, DPINN_ERR_STATE, "point set not present");
  const std::vector<int64_t>& cnt = kind == 0 ? h->res_counts : (kind == 1 ? h->obs_counts : h->face_counts);
  int64_t n = 0;
  for (int64_t c : cnt) n += c;
  const DevBuf<float>& pb = kind == 0 ? h->res_pts : (kind == 1 ? h->obs_pts : h->face_pts);
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaDeviceSynchronize());
  if (n) CK(h, cudaMemcpy(host_out, pb.p, (size_t)n * h->din * sizeof(float), cudaMemcpyDeviceToHost));
  return DPINN_OK;
}

int dpinn_set_partial_budget(dpinn_t* h, int64_t bytes) {
  if (!h || bytes < 0) return DPINN_ERR_INVALID_ARG;
  const int64_t b = bytes ? bytes : ((int64_t)1 << 30);
  if (b == h->part_budget) return DPINN_OK;
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaDeviceSynchronize());
  h->part_budget = b;
  h->plan_ok = false;
  return build_plan(h);
}

int dpinn_step(dpinn_t* h, dpinn_stream_t stream, int n_steps) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (!h->plan_ok) {
    int rc = build_plan(h);
    if (rc) return rc;
    if (!h->plan_ok) return fail(h, DPINN_ERR_STATE, "residual, observation and face points must be set first");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = apply_stage(h, s)) return rc;
  for (int i = 0; i < n_steps; ++i) CK(h, cudaGraphLaunch(h->g_step, s));
  CK(h, cudaEventRecord(h->done, s));
  return DPINN_OK;
}

int dpinn_eval_grad(dpinn_t* h, dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (!h->plan_ok) {
    int rc = build_plan(h);
    if (rc) return rc;
    if (!h->plan_ok) return fail(h, DPINN_ERR_STATE, "residual, observation and face points must be set first");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = apply_stage(h, s)) return rc;
  CK(h, cudaGraphLaunch(h->g_grad, s));
  CK(h, cudaEventRecord(h->done, s));
  return DPINN_OK;
}

int dpinn_eval_loss(dpinn_t* h, dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (!h->plan_ok) {
    int rc = build_plan(h);
    if (rc) return rc;
    if (!h->plan_ok) return fail(h, DPINN_ERR_STATE, "residual, observation and face points must be set first");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = apply_stage(h, s)) return rc;
  CK(h, cudaGraphLaunch(h->g_loss, s));
  CK(h, cudaEventRecord(h->done, s));
  return DPINN_OK;
}

int dpinn_set_schedule(dpinn_t* h, int jet_tiles, int val_tiles, int order) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (jet_tiles < 0 || jet_tiles > 4096 || val_tiles < 0 || val_tiles > 4096 || order < 0 || order > 1)
    return fail(h, DPINN_ERR_INVALID_ARG, "bad schedule");
  if (jet_tiles == h->sched_jet && val_tiles == h->sched_val && order == h->sched_order) return DPINN_OK;
  CK(h, cudaDeviceSynchronize());
  h->sched_jet = jet_tiles;
  h->sched_val = val_tiles;
  h->sched_order = order;
  return build_plan(h);
}

int dpinn_set_precision(dpinn_t* h, int precision) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (precision != DPINN_PREC_FP32 && precision != DPINN_PREC_TF32X3)
    return fail(h, DPINN_ERR_INVALID_ARG, "precision must be FP32 or TF32x3");
  if (precision == DPINN_PREC_TF32X3 && h->W != 128)
    return fail(h, DPINN_ERR_INVALID_ARG, "TF32x3 tensor-core kernels need width 128");
  if (precision == DPINN_PREC_TF32X3)
    for (int l = 1; l < h->L; ++l)
      if (h->shape.woff[l] % 4 != 0) return fail(h, DPINN_ERR_INVALID_ARG, "weight-gradient tile not 16-byte aligned");
  if (precision == h->cfg.precision) return DPINN_OK;
  CK(h, cudaDeviceSynchronize());
  if (int rc = select_kernels(h, precision)) return rc;
  return build_plan(h);
}

int dpinn_tile_options(dpinn_t* h, int* jet_points, int* n_jet, int* val_points, int* n_val) {
  if (!h || !jet_points || !n_jet || !val_points || !n_val) return DPINN_ERR_INVALID_ARG;
  if (h->cfg.precision == DPINN_PREC_TF32X3) {
    jet_points[0] = h->ks.P_tc;
    val_points[0] = h->ks.P_tcv;
    *n_jet = *n_val = 1;
    return DPINN_OK;
  }
  jet_points[0] = h->ks.P_jet;
  val_points[0] = h->ks.P_val;
  *n_jet = *n_val = 1;
  if (h->ks.train_jet_alt) jet_points[(*n_jet)++] = h->ks.P_jet_alt;
  if (h->ks.train_val_alt) val_points[(*n_val)++] = h->ks.P_val_alt;
  return DPINN_OK;
}

int dpinn_set_tiles(dpinn_t* h, int jet_tile, int val_tile) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  int jo[2], vo[2], nj = 0, nv = 0;
  dpinn_tile_options(h, jo, &nj, vo, &nv);
  if (jet_tile < 0 || jet_tile >= nj || val_tile < 0 || val_tile >= nv)
    return fail(h, DPINN_ERR_INVALID_ARG, "tile index not available (see dpinn_tile_options)");
  if (h->cfg.precision == DPINN_PREC_TF32X3) return DPINN_OK;   // one tile per tensor-core kernel
  if (jet_tile == h->tile_jet && val_tile == h->tile_val) return DPINN_OK;
  CK(h, cudaDeviceSynchronize());
  h->tile_jet = jet_tile;
  h->tile_val = val_tile;
  if (int rc = select_kernels(h, h->cfg.precision)) return rc;
  return build_plan(h);
}

int dpinn_get_tiles(dpinn_t* h, int* jet_tile, int* val_tile) {
  if (!h || !jet_tile || !val_tile) return DPINN_ERR_INVALID_ARG;
  const bool tc = h->cfg.precision == DPINN_PREC_TF32X3;
  *jet_tile = tc ? 0 : h->tile_jet;
  *val_tile = tc ? 0 : h->tile_val;
  return DPINN_OK;
}

int dpinn_get_precision(dpinn_t* h, int* precision) {
  if (!h || !precision) return DPINN_ERR_INVALID_ARG;
  *precision = h->cfg.precision;
  return DPINN_OK;
}

int dpinn_get_schedule(dpinn_t* h, int* jet_tiles, int* val_tiles, int* order, int* tile_points) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (jet_tiles) *jet_tiles = h->sched_jet;
  if (val_tiles) *val_tiles = h->sched_val;
  if (order) *order = h->sched_order;
  if (tile_points) { tile_points[0] = h->ks.P_train_jet; tile_points[1] = h->ks.P_val_run; }
  return DPINN_OK;
}

int dpinn_set_params(dpinn_t* h, const float* params) {
  if (!h || !params) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaDeviceSynchronize());
  int rc = copy_state_in(h, h->theta.p, params);
  if (rc) return rc;
  return refresh_transpose(h);
}

int dpinn_loss(dpinn_t* h, float* host_out) {
  if (!h || !host_out) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaEventSynchronize(h->done));
  // the first 6 of the 8 entries per net
  CK(h, cudaMemcpy2D(host_out, 6 * sizeof(float), h->loss_rec.p, 8 * sizeof(float), 6 * sizeof(float), h->n_nets,
                     cudaMemcpyDeviceToHost));
  return check_errors(h);
}

int dpinn_loss_async(dpinn_t* h, float* host_out, dpinn_stream_t stream) {
  if (!h || !host_out) return DPINN_ERR_INVALID_ARG;
  // the first 6 of the 8 entries per net, in stream order after the step
  CK(h, cudaMemcpy2DAsync(host_out, 6 * sizeof(float), h->loss_rec.p, 8 * sizeof(float), 6 * sizeof(float),
                          h->n_nets, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  return DPINN_OK;
}

int dpinn_loss_ext(dpinn_t* h, float* host_out) {
  if (!h || !host_out) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaEventSynchronize(h->done));
  CK(h, cudaMemcpy(host_out, h->loss_rec.p, (size_t)h->n_nets * 8 * sizeof(float), cudaMemcpyDeviceToHost));
  return check_errors(h);
}

int dpinn_get_grad(dpinn_t* h, float* host_out) {
  if (!h || !host_out) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaEventSynchronize(h->done));
  return copy_state_out(h, host_out, h->grad.p);
}

int dpinn_get_state(dpinn_t* h, float* params, float* m, float* v, int64_t* step) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaDeviceSynchronize());
  int rc = DPINN_OK;
  if (params && (rc = copy_state_out(h, params, h->theta.p))) return rc;
  if (m && (rc = copy_state_out(h, m, h->m.p))) return rc;
  if (v && (rc = copy_state_out(h, v, h->v.p))) return rc;
  if (step) {
    long long t = 0;
    CK(h, cudaMemcpy(&t, h->step_d.p, sizeof(t), cudaMemcpyDeviceToHost));
    *step = t;
  }
  return DPINN_OK;
}

int dpinn_set_state(dpinn_t* h, const float* params, const float* m, const float* v, int64_t step) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (step < 0) return fail(h, DPINN_ERR_INVALID_ARG, "negative step");
  CK(h, cudaDeviceSynchronize());
  int rc = DPINN_OK;
  if (params && (rc = copy_state_in(h, h->theta.p, params))) return rc;
  if (m && (rc = copy_state_in(h, h->m.p, m))) return rc;
  if (v && (rc = copy_state_in(h, h->v.p, v))) return rc;
  long long t = step;
  CK(h, cudaMemcpy(h->step_d.p, &t, sizeof(t), cudaMemcpyHostToDevice));
  return refresh_transpose(h);
}

int dpinn_apply_grad(dpinn_t* h, const float* host_grad) {
  if (!h || !host_grad) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaDeviceSynchronize());
  int rc = copy_state_in(h, h->grad.p, host_grad);
  if (rc) return rc;
  const int nblk = (h->n_params + dk::NT - 1) / dk::NT;
  // per-net norms of the given gradient (slot k = net k of the grad buffer)
  dk::k_reduce_grad<<<dim3(nblk, h->n_nets), dk::NT>>>(h->grad.p, h->iota_d.p, h->grad.p, h->norm_part.p, h->npp,
                                                        h->n_params);
  if (h->cfg.clip_norm > 0)
    dk::k_clip_coef<<<h->n_nets, dk::NT>>>(h->norm_part.p, nblk, (float)h->cfg.clip_norm, h->coef.p);
  const dk::AdamArgs ar = adam_args(h);
  dk::k_adam<<<dim3(nblk, h->n_nets), dk::NT>>>(h->shape, ar, h->theta.p, h->thetaT.p, h->m.p, h->v.p, h->grad.p,
                                                 h->coef.p, h->step_d.p, h->n_params);
  dk::k_loss_record<<<1, 32>>>(h->shape, h->loss_part.p, h->slot_begin_d.p, h->nets_d.p, 0, h->loss_rec.p,
                                h->err_d.p, h->step_d.p, 1);
  CK(h, cudaGetLastError());
  CK(h, cudaDeviceSynchronize());
  return DPINN_OK;
}

int dpinn_query(dpinn_t* h, const float* pts, int64_t n, int want_residual, float* out, dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  return handle_query(h, pts, n, want_residual ? Q_RESIDUAL : Q_VALUES, out, (cudaStream_t)stream);
}

int dpinn_query_jets(dpinn_t* h, const float* pts, int64_t n, float* out, dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  return handle_query(h, pts, n, Q_JETS, out, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
// Scratch of dpinn_query_static: one fixed-size array in device memory,
// reserved on every GPU that loads this library until the process exits.
// Layout (byte offsets, each part 256-byte aligned): the net of each point,
// the points ordered by net, per-net counts / segment starts / scatter
// cursors, the work-item count, the work items.
constexpr int64_t QS_MAX_POINTS = 262144;
constexpr int QS_MAX_NETS = 4096;
constexpr int QS_MAX_ITEMS = (int)(QS_MAX_POINTS / 64) + QS_MAX_NETS + 1;   // chunks are >= 64 points
constexpr size_t QS_OFF_NET = 0;
constexpr size_t QS_OFF_PERM = QS_OFF_NET + QS_MAX_POINTS * sizeof(int);
constexpr size_t QS_OFF_COUNTS = QS_OFF_PERM + QS_MAX_POINTS * sizeof(int);
constexpr size_t QS_OFF_OFFSETS = QS_OFF_COUNTS + QS_MAX_NETS * sizeof(int);
constexpr size_t QS_OFF_CURSOR = QS_OFF_OFFSETS + QS_MAX_NETS * sizeof(int);
constexpr size_t QS_OFF_NITEMS = QS_OFF_CURSOR + QS_MAX_NETS * sizeof(int);
constexpr size_t QS_OFF_ITEMS = QS_OFF_NITEMS + 256;
constexpr size_t QS_BYTES = QS_OFF_ITEMS + (size_t)QS_MAX_ITEMS * sizeof(dk::Item);

static __device__ __align__(256) unsigned char g_query_scratch[QS_BYTES];

// Device address of g_query_scratch per device ordinal, looked up once per
// device (the symbol's host-side name is not a device address).  The cache
// lives as long as the process; it does not survive a device reset or a
// teardown of the device's primary context (nor does the library's module).
std::mutex g_qs_mu;
void* g_qs_addr[256] = {nullptr};

int query_scratch_address(dpinn* h, void** out) {
  std::lock_guard<std::mutex> lock(g_qs_mu);
  if (h->dev < 0 || h->dev >= 256) return fail(h, DPINN_ERR_INVALID_ARG, "device ordinal out of range");
  if (!g_qs_addr[h->dev]) {
    int cur = 0;
    CK(h, cudaGetDevice(&cur));
    if (cur != h->dev) CK(h, cudaSetDevice(h->dev));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_query_scratch);
    if (cur != h->dev) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress(g_query_scratch)");
    g_qs_addr[h->dev] = p;
  }
  *out = g_qs_addr[h->dev];
  return DPINN_OK;
}
}  // namespace

extern "C" {

int dpinn_query_static(dpinn_t* h, const float* pts, int64_t n, int want_residual, float* out,
                       dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  if (n < 0 || n > QS_MAX_POINTS)
    return fail(h, DPINN_ERR_INVALID_ARG, "dpinn_query_static serves at most 262144 points per call");
  if (h->n_nets > QS_MAX_NETS)
    return fail(h, DPINN_ERR_INVALID_ARG, "dpinn_query_static serves ensembles of at most 4096 nets");
  if (n == 0) return DPINN_OK;
  if (!pts || !out) return fail(h, DPINN_ERR_INVALID_ARG, "null pointer");
  const int mode = want_residual ? Q_RESIDUAL : Q_VALUES;
  // every work item must fit the fixed array (holds while query tiles have
  // at least 16 points); refused before anything is launched
  if (query_max_items(h, n, mode) > (size_t)QS_MAX_ITEMS)
    return fail(h, DPINN_ERR_STATE, "dpinn_query_static: work items exceed the fixed array");
  void* base = nullptr;
  int rc = query_scratch_address(h, &base);
  if (rc) return rc;
  char* sb = static_cast<char*>(base);
  // the array keeps the previous call's contents; enqueue_query clears the
  // counters it accumulates into (per-net counts, item count) on the stream
  QueryScratch qs{reinterpret_cast<int*>(sb + QS_OFF_NET),     reinterpret_cast<int*>(sb + QS_OFF_PERM),
                  reinterpret_cast<int*>(sb + QS_OFF_COUNTS),  reinterpret_cast<int*>(sb + QS_OFF_OFFSETS),
                  reinterpret_cast<int*>(sb + QS_OFF_CURSOR),  reinterpret_cast<int*>(sb + QS_OFF_NITEMS),
                  reinterpret_cast<dk::Item*>(sb + QS_OFF_ITEMS), h->err_d.p, (size_t)QS_MAX_ITEMS};
  return enqueue_query(h, qs, pts, n, mode, out, (cudaStream_t)stream);
}

int dpinn_qctx_create(dpinn_t* h, int64_t max_points, dpinn_qctx_t** out) {
  if (!h || !out) return DPINN_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_points < 1 || max_points > ((int64_t)1 << 30)) return fail(h, DPINN_ERR_INVALID_ARG, "bad max_points");
  std::unique_ptr<dpinn_qctx> q(new dpinn_qctx());
  q->h = h;
  q->cap = max_points;
  const int Pmin = std::min(h->ks.P_qjet, h->ks.P_qval);
  q->items_cap = (size_t)(max_points / (4 * Pmin)) + h->n_nets + 1;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sz[8] = {(size_t)max_points * 4, (size_t)max_points * 4, (size_t)h->n_nets * 4,
                        (size_t)h->n_nets * 4, (size_t)h->n_nets * 4, 2 * 4, 4 * 4,
                        q->items_cap * sizeof(dk::Item)};
  size_t off[8], total = 0;
  for (int i = 0; i < 8; ++i) { off[i] = total; total += up(sz[i]); }
  CK(h, q->mem.ensure(total));
  unsigned char* b = q->mem.p;
  q->net_of = reinterpret_cast<int*>(b + off[0]);
  q->perm = reinterpret_cast<int*>(b + off[1]);
  q->counts = reinterpret_cast<int*>(b + off[2]);
  q->offsets = reinterpret_cast<int*>(b + off[3]);
  q->cursor = reinterpret_cast<int*>(b + off[4]);
  q->nitems = reinterpret_cast<int*>(b + off[5]);
  q->err = reinterpret_cast<int*>(b + off[6]);
  q->items = reinterpret_cast<dk::Item*>(b + off[7]);
  CK(h, cudaMemset(q->err, 0, 4 * sizeof(int)));
  *out = q.release();
  return DPINN_OK;
}

void dpinn_qctx_destroy(dpinn_qctx_t* q) {
  if (!q) return;
  cudaSetDevice(q->h->dev);
  cudaDeviceSynchronize();
  delete q;
}

int dpinn_qctx_query(dpinn_qctx_t* q, const float* pts, int64_t n, int want_residual, float* out,
                     dpinn_stream_t stream) {
  if (!q) return DPINN_ERR_INVALID_ARG;
  dpinn* h = q->h;
  if (n < 0 || n > q->cap) return fail(h, DPINN_ERR_INVALID_ARG, "more points than the context was created for");
  if (n == 0) return DPINN_OK;
  if (!pts || !out) return fail(h, DPINN_ERR_INVALID_ARG, "null pointer");
  QueryScratch qs{q->net_of, q->perm, q->counts, q->offsets, q->cursor, q->nitems, q->items, q->err, q->items_cap};
  return enqueue_query(h, qs, pts, n, want_residual ? Q_RESIDUAL : Q_VALUES, out, (cudaStream_t)stream);
}

int dpinn_qctx_status(dpinn_qctx_t* q, dpinn_stream_t stream) {
  if (!q) return DPINN_ERR_INVALID_ARG;
  dpinn* h = q->h;
  CK(h, cudaStreamSynchronize((cudaStream_t)stream));
  int e[3] = {0, 0, 0};
  CK(h, cudaMemcpy(e, q->err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e[dk::ERR_TIMEOUT]) return fail(h, DPINN_ERR_TIMEOUT, "a device wait gave up");
  if (e[dk::ERR_DOMAIN]) {
    CK(h, cudaMemset(q->err + dk::ERR_DOMAIN, 0, sizeof(int)));
    return fail(h, DPINN_ERR_INVALID_ARG, "query point outside the domain");
  }
  return DPINN_OK;
}

int dpinn_query_status(dpinn_t* h, dpinn_stream_t stream) {
  if (!h) return DPINN_ERR_INVALID_ARG;
  CK(h, cudaStreamSynchronize((cudaStream_t)stream));
  int e[3] = {0, 0, 0};
  CK(h, cudaMemcpy(e, h->err_d.p, sizeof(e), cudaMemcpyDeviceToHost));
  if (e[dk::ERR_TIMEOUT]) return fail(h, DPINN_ERR_TIMEOUT, "a device wait gave up");
  if (e[dk::ERR_DOMAIN]) {
    CK(h, cudaMemset(h->err_d.p + dk::ERR_DOMAIN, 0, sizeof(int)));
    return fail(h, DPINN_ERR_INVALID_ARG, "query point outside the domain");
  }
  return DPINN_OK;
}

int dpinn_launches_per_step(dpinn_t* h) { return h ? h->launches : 0; }

int dpinn_step_timed(dpinn_t* h, dpinn_stream_t stream, float* ms, int max_kernels, int* n_kernels,
                     const char** names) {
  if (!h || !ms || max_kernels < 1) return DPINN_ERR_INVALID_ARG;
  if (!h->plan_ok) {
    int rc = build_plan(h);
    if (rc) return rc;
    if (!h->plan_ok) return fail(h, DPINN_ERR_STATE, "residual, observation and face points must be set first");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = apply_stage(h, s)) return rc;
  cudaEvent_t ev[12];   // at most 8 kernels per step
  for (auto& e : ev) CK(h, cudaEventCreate(&e));
  const char* nm[11] = {nullptr};
  int launches = 0;
  cudaError_t e = enqueue_step(h, RUN_STEP, s, &launches, ev, nm);
  if (e == cudaSuccess) e = cudaEventRecord(h->done, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[launches]);
  const int n = std::min(launches, max_kernels);
  for (int i = 0; e == cudaSuccess && i < n; ++i) {
    e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    if (names) names[i] = nm[i];
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(h, e, "dpinn_step_timed");
  if (n_kernels) *n_kernels = n;
  return DPINN_OK;
}

}  // extern "C"

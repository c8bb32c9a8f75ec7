// Kernel sets of the grouped kernel k_pinn: one translation unit per width
// and activation instantiates them (kernels_w*_*.cu), so that the many
// instantiations compile in parallel.
#pragma once
#include <cstddef>

namespace dk {

struct KernelSet {
  const void* train_jet = nullptr;
  const void* train_val = nullptr;
  const void* eval_val = nullptr;
  const void* eval_jet = nullptr;   // exchange with jets (interface residual / C1 terms)
  const void* query_val = nullptr;
  const void* query_jet = nullptr;
  size_t smem_jet = 0, smem_val = 0;
  int P_jet = 0, P_val = 0;
  long long stash_jet = 0, stash_val = 0;   // floats per CTA
  // alternate point tiles of the FP32 jet training kernel and of the value
  // training / exchange kernels (null where the family has none)
  const void* train_jet_alt = nullptr;
  const void* train_val_alt = nullptr;
  const void* eval_val_alt = nullptr;
  size_t smem_jet_alt = 0, smem_val_alt = 0;
  int P_jet_alt = 0, P_val_alt = 0;
  long long stash_jet_alt = 0, stash_val_alt = 0;
  // the jet training kernel actually launched (the FP32 one above, or the
  // tensor-core one below), its shared memory, tile and stash
  const void* train_jet_run = nullptr;
  int threads_train_jet = 0;
  size_t smem_train_jet = 0;
  int P_train_jet = 0;
  long long stash_train_jet = 0;
  // tensor-core (tcgen05, 3xTF32) jet training kernel, width 128 only
  const void* train_jet_tc = nullptr;
  int threads_tc = 0;
  size_t smem_tc = 0;
  int P_tc = 0;
  long long stash_tc = 0;
  // the value kernels actually launched (training of observation / face
  // items, and the exchange): FP32 ones above or the tensor-core ones below
  const void* train_val_run = nullptr;
  const void* eval_val_run = nullptr;
  int threads_val_run = 0, P_val_run = 0;
  size_t smem_val_run = 0;
  long long stash_val_run = 0;
  // tensor-core value kernels, width 128 only
  const void* train_val_tc = nullptr;
  const void* eval_val_tc = nullptr;
  const void* query_val_tc = nullptr;
  const void* query_jet_tc = nullptr;
  // the query kernels actually launched and their launch shapes
  const void* query_val_run = nullptr;
  const void* query_jet_run = nullptr;
  int threads_qval = 0, threads_qjet = 0, P_qval = 0, P_qjet = 0;
  size_t smem_qval = 0, smem_qjet = 0;
  int threads_tcv = 0;
  size_t smem_tcv = 0;
  int P_tcv = 0;
  long long stash_tcv = 0;
};

// Fill *k for (d_space, unsteady, depth); false if the shape is unsupported.
bool kernels_w32_tanh(int ds, int unst, int L, KernelSet* k);
bool kernels_w64_tanh(int ds, int unst, int L, KernelSet* k);
bool kernels_w128_tanh(int ds, int unst, int L, KernelSet* k);
bool kernels_w32_sin(int ds, int unst, int L, KernelSet* k);
bool kernels_w64_sin(int ds, int unst, int L, KernelSet* k);
bool kernels_w128_sin(int ds, int unst, int L, KernelSet* k);
// other widths (the cylinder networks: 150, 200): the streamed-weight kernel
// k_pinn_w, padded to 160 (widths 129-160) or 224 (161-224)
bool kernels_wide160_tanh(int ds, int unst, int L, KernelSet* k);
bool kernels_wide160_sin(int ds, int unst, int L, KernelSet* k);
bool kernels_wide224_tanh(int ds, int unst, int L, KernelSet* k);
bool kernels_wide224_sin(int ds, int unst, int L, KernelSet* k);

}  // namespace dk

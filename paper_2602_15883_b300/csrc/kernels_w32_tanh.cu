// Instantiates the grouped kernels for width 32 with the tanh activation.
#include "kernel_set.h"
#include "pinn_kernels.cuh"

namespace dk {
namespace {

template <int W, int DS, int UNST, int ACT>
KernelSet make_set(int L) {
  constexpr int DIN = DS + UNST, CJ = DIN + 2, DOUT = DS + 1;
  KernelSet k;
  k.train_jet = (const void*)k_pinn<W, DS, UNST, true, M_TRAIN, ACT>;
  k.train_val = (const void*)k_pinn<W, DS, UNST, false, M_TRAIN, ACT>;
  k.eval_val = (const void*)k_pinn<W, DS, UNST, false, M_EVAL, ACT>;
  k.eval_jet = (const void*)k_pinn<W, DS, UNST, true, M_EVAL, ACT>;
  k.query_val = (const void*)k_pinn<W, DS, UNST, false, M_QUERY, ACT>;
  k.query_jet = (const void*)k_pinn<W, DS, UNST, true, M_QUERY, ACT>;
  k.smem_jet = smem_floats<W, CJ, DOUT>(L) * sizeof(float);
  k.smem_val = smem_floats<W, 1, DOUT>(L) * sizeof(float);
  k.P_jet = Tile<W, CJ>::P;
  k.P_val = Tile<W, 1>::P;
  k.stash_jet = (long long)L * Tile<W, CJ>::NQ * NT * 4;
  k.stash_val = (long long)L * Tile<W, 1>::NQ * NT * 4;
  if constexpr (Tile<W, CJ, 1>::P != Tile<W, CJ>::P || Tile<W, CJ, 1>::TM != Tile<W, CJ>::TM) {
    k.train_jet_alt = (const void*)k_pinn<W, DS, UNST, true, M_TRAIN, ACT, 1>;
    k.smem_jet_alt = smem_floats<W, CJ, DOUT, 1>(L) * sizeof(float);
    k.P_jet_alt = Tile<W, CJ, 1>::P;
    k.stash_jet_alt = (long long)L * Tile<W, CJ, 1>::NQ * NT * 4;
  }
  if constexpr (Tile<W, 1, 1>::P != Tile<W, 1>::P || Tile<W, 1, 1>::TM != Tile<W, 1>::TM) {
    k.train_val_alt = (const void*)k_pinn<W, DS, UNST, false, M_TRAIN, ACT, 1>;
    k.eval_val_alt = (const void*)k_pinn<W, DS, UNST, false, M_EVAL, ACT, 1>;
    k.smem_val_alt = smem_floats<W, 1, DOUT, 1>(L) * sizeof(float);
    k.P_val_alt = Tile<W, 1, 1>::P;
    k.stash_val_alt = (long long)L * Tile<W, 1, 1>::NQ * NT * 4;
  }
  return k;
}

}  // namespace

bool kernels_w32_tanh(int ds, int unst, int L, KernelSet* k) {
  if (ds == 2 && unst == 0) { *k = make_set<32, 2, 0, ACT_TANH>(L); return true; }
  if (ds == 2 && unst == 1) { *k = make_set<32, 2, 1, ACT_TANH>(L); return true; }
  if (ds == 3 && unst == 0) { *k = make_set<32, 3, 0, ACT_TANH>(L); return true; }
  if (ds == 3 && unst == 1) { *k = make_set<32, 3, 1, ACT_TANH>(L); return true; }
  return false;
}

}  // namespace dk

// Instantiates the wide grouped kernels (widths 193..224, padded to 224) with the sin activation.
#include "kernel_set.h"
#include "pinn_wide.cuh"

namespace dk {
namespace {

template <int WP, int DS, int UNST, int ACT>
KernelSet make_set(int L) {
  constexpr int DIN = DS + UNST, CJ = DIN + 2, DOUT = DS + 1;
  KernelSet k;
  k.train_jet = (const void*)k_pinn_w<WP, DS, UNST, true, M_TRAIN, ACT>;
  k.train_val = (const void*)k_pinn_w<WP, DS, UNST, false, M_TRAIN, ACT>;
  k.eval_val = (const void*)k_pinn_w<WP, DS, UNST, false, M_EVAL, ACT>;
  k.eval_jet = (const void*)k_pinn_w<WP, DS, UNST, true, M_EVAL, ACT>;
  k.query_val = (const void*)k_pinn_w<WP, DS, UNST, false, M_QUERY, ACT>;
  k.query_jet = (const void*)k_pinn_w<WP, DS, UNST, true, M_QUERY, ACT>;
  k.smem_jet = smem_floats_wide<WP, CJ, DOUT>(L) * sizeof(float);
  k.smem_val = smem_floats_wide<WP, 1, DOUT>(L) * sizeof(float);
  k.P_jet = WideTile<WP, CJ>::P;
  k.P_val = WideTile<WP, 1>::P;
  k.stash_jet = (long long)L * WideTile<WP, CJ>::NQ * NTW;
  k.stash_val = (long long)L * WideTile<WP, 1>::NQ * NTW;
  k.train_jet_alt = (const void*)k_pinn_w<WP, DS, UNST, true, M_TRAIN, ACT, 1>;
  k.smem_jet_alt = smem_floats_wide<WP, CJ, DOUT, 1>(L) * sizeof(float);
  k.P_jet_alt = WideTile<WP, CJ, 1>::P;
  k.stash_jet_alt = (long long)L * WideTile<WP, CJ, 1>::NQ * NTW;
  k.train_val_alt = (const void*)k_pinn_w<WP, DS, UNST, false, M_TRAIN, ACT, 1>;
  k.eval_val_alt = (const void*)k_pinn_w<WP, DS, UNST, false, M_EVAL, ACT, 1>;
  k.smem_val_alt = smem_floats_wide<WP, 1, DOUT, 1>(L) * sizeof(float);
  k.P_val_alt = WideTile<WP, 1, 1>::P;
  k.stash_val_alt = (long long)L * WideTile<WP, 1, 1>::NQ * NTW;
  return k;
}

}  // namespace

bool kernels_wide224_sin(int ds, int unst, int L, KernelSet* k) {
  if (ds == 2 && unst == 0) { *k = make_set<224, 2, 0, ACT_SIN>(L); return true; }
  if (ds == 2 && unst == 1) { *k = make_set<224, 2, 1, ACT_SIN>(L); return true; }
  if (ds == 3 && unst == 0) { *k = make_set<224, 3, 0, ACT_SIN>(L); return true; }
  if (ds == 3 && unst == 1) { *k = make_set<224, 3, 1, ACT_SIN>(L); return true; }
  return false;
}

}  // namespace dk

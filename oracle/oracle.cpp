// FP64 CPU oracle for one training step of the domain-decomposed PINN
// (arXiv 2602.15883, "Distributed physics-informed neural networks via domain
// decomposition for fast flow reconstruction").
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
// the benchmark's CPU-baseline leg load this library.  It shares no code,
// header, table or constant with the CUDA path: it restates the paper's
// definitions in plain double-precision loops so that a reader can check it
// against the paper by eye.  No blocking, fusion or reordering beyond what the
// definitions state.
//
// What it follows (equation numbers count the paper's numbered equations in
// order of appearance):
//   * network (u, p) = NN(x, t; theta), fully connected tanh MLP,
//     or sin for the cylinder cases                               - Sec. 2.1, Eq. (2); Sec. 5
//   * L_obs, mean over points of ||u_obs - u_NN||_2^2             - Eq. (3)
//   * L_PDE, mean over points of ||r||_2^2                         - Eq. (5)
//   * incompressible Navier-Stokes residuals r_1..r_4, 1/Re = nu   - Eqs. (6)-(10)
//   * K x M space-time decomposition, one independent net each     - Sec. 2.2
//   * ghost consistency losses L_gh_u, L_gh_p against cached
//     (constant) neighbour predictions                             - Eqs. (13)-(14)
//   * master ranks: nets whose spatial cell holds x_anc            - Sec. 2.2, Algorithm 1
//   * anchor normalisation p~ = p(x,t) - p(x_anc,t), only on the
//     pressure a master sends                                      - Eq. (15), Algorithm 1
//   * decoupled asymmetric weighting: lambda^space = 0 on masters,
//     lambda^time > 0 everywhere                                   - Sec. 2.2 (1)-(2), Eq. (16)
//   * local objective L_{k,m}                                      - Eq. (16)
//   * one optimiser step per iteration (Adam)                      - Algorithm 1
//   * anchored pressure for output of master cells                 - Sec. 3, Eq. (18)
//   * volumetric ghost layers of thickness delta (ghost points of A
//     evaluated by the net whose cell holds them)                  - Sec. 2.2
//   * interface residual and C1 matching terms on ghost points     - Remark, Sec. 2.2
//   * messages refreshed every I_comm iterations, stale between    - Algorithm 1
//   * step decay of the learning rate (factor, interval)           - Table B1
//   * per-step uniform resampling of collocation points from
//     counter-based SplitMix64 streams                             - Sec. 3 (epochs)
//
// Readings where the paper is silent (each listed in the design notes):
//   * inputs are mapped from the net's own interior box to [-1, 1];
//   * ghost points are shared face points (zero-thickness ghost layer);
//     L_gh terms of net A are divided by the total number of points on A's
//     faces, and split into spatial and temporal parts by face type;
//   * the anchor is evaluated at each ghost point's own time;
//   * the exchange uses values at the current parameters (I_comm = 1);
//   * component weights w_c multiply velocity components in L_obs and L_gh_u;
//   * the optimiser is Adam with PyTorch's update rule, optional per-net
//     gradient-norm clipping with coefficient min(1, c / (||g|| + 1e-6)).
//
// Parity status: every function here is pinned by the CPU tests (complex-step
// and finite differences, analytic flows, invariants, closed forms, PyTorch
// FP64 double backward); none is "parity unpinned".
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

// ---------------------------------------------------------------- config ---
struct ora_config {
  int d_space, unsteady, depth, width;
  int splits[4];
  double lo[4], hi[4];
  double nu;
  double anchor[3];
  double p_ref;
  double lam_obs, lam_pde, lam_gh_u, lam_gh_p_space, lam_gh_p_time;
  double comp_w[3];
  double lr, beta1, beta2, eps, clip;
  double lr_decay_factor;   // update t uses lr * factor^floor((t-1)/interval)
  int lr_decay_interval;    // 0: constant learning rate
  int comm_interval;        // Algorithm 1: messages refreshed when t mod I_comm == 0
  int activation;           // 0 tanh, 1 sin
  // Interface terms beyond C0 (Remark, Sec. 2.2), 0 = off: residual matching
  // sum_j (r_A - sg r_B)_j^2 and C1 matching sum_{c,q} (d_q Y_A,c - sg d_q Y_B,c)^2
  // at the ghost points, divided by N_gh like Eqs. (13)-(14).
  double lam_gh_r, lam_gh_c1;
};

struct ora_problem {
  const float* res_pts;  const int64_t* res_counts;   // [n_res][d_in], [n_nets]
  const float* obs_pts;  const float* obs_vals;       // [n_obs][d_in], [n_obs][d_space]
  const int64_t* obs_counts;                          // [n_nets]
  const float* face_pts; const int64_t* face_counts;  // [n_face][d_in], [n_faces]
  // Volumetric ghost layers (delta > 0): points of each net outside its own
  // cell; when ghost_counts is set they replace the face points.
  const float* ghost_pts; const int64_t* ghost_counts;  // [n_ghost][d_in], [n_nets]
};


namespace {

using cplx = std::complex<double>;

int g_threads = 1;

// Cell of coordinate x along axis a, decided in FP32 exactly as the library's
// routing rule states it: floor((x - lo) * (splits / (hi - lo))) with every
// operation rounded to float, clamped to the valid range.  Returns -1 when x
// lies outside [lo, hi].
int cell_fp32(const ora_config& c, int a, float x) {
  volatile float lo = (float)c.lo[a];
  volatile float hi = (float)c.hi[a];
  volatile float inv_h = (float)((double)c.splits[a] / (c.hi[a] - c.lo[a]));
  if (!(x >= lo && x <= hi)) return -1;
  volatile float d = x - lo;
  volatile float q = d * inv_h;
  int k = (int)std::floor((float)q);
  if (k < 0) k = 0;
  if (k > c.splits[a] - 1) k = c.splits[a] - 1;
  return k;
}

// ---------------------------------------------------------------- layout ---
struct Geo {
  ora_config cfg;
  int ds, unst, din, dout, C, LAP, L, W, n_nets, n_faces, n_params;
  std::vector<int> stride;
  std::vector<std::array<int, 4>> cell;
  std::vector<std::array<double, 4>> blo, bhi;
  std::vector<int> master;
  std::vector<std::array<int, 3>> face;       // lo net, hi net, axis
  std::vector<int> woff, boff, nout, nin;     // per affine map l = 0..L
  std::vector<std::vector<std::pair<int, int>>> net_faces;  // (face, side)

  explicit Geo(const ora_config& c) : cfg(c) {
    ds = c.d_space; unst = c.unsteady; din = ds + unst; dout = ds + 1;
    C = din + 2; LAP = din + 1; L = c.depth; W = c.width;
    n_nets = 1;
    for (int a = 0; a < din; ++a) { stride.push_back(n_nets); n_nets *= c.splits[a]; }
    for (int k = 0; k < n_nets; ++k) {
      std::array<int, 4> ce{0, 0, 0, 0};
      std::array<double, 4> lo{0, 0, 0, 0}, hi{0, 0, 0, 0};
      int r = k;
      for (int a = 0; a < din; ++a) {
        ce[a] = r % c.splits[a]; r /= c.splits[a];
        double h = (c.hi[a] - c.lo[a]) / c.splits[a];
        lo[a] = c.lo[a] + ce[a] * h;
        hi[a] = c.lo[a] + (ce[a] + 1) * h;
      }
      cell.push_back(ce); blo.push_back(lo); bhi.push_back(hi);
    }
    // Algorithm 1: masters are the nets whose spatial cell contains x_anc,
    // for every time slab.
    int acell[3] = {0, 0, 0};
    for (int a = 0; a < ds; ++a) acell[a] = cell_fp32(c, a, (float)c.anchor[a]);
    for (int k = 0; k < n_nets; ++k) {
      bool m = true;
      for (int a = 0; a < ds; ++a) m = m && (cell[k][a] == acell[a]);
      master.push_back(m ? 1 : 0);
    }
    // Faces between neighbouring cells, axis by axis, lower net ascending.
    net_faces.resize(n_nets);
    for (int a = 0; a < din; ++a)
      for (int k = 0; k < n_nets; ++k)
        if (cell[k][a] < c.splits[a] - 1) {
          int f = (int)face.size();
          face.push_back({k, k + stride[a], a});
          net_faces[k].push_back({f, 0});
          net_faces[k + stride[a]].push_back({f, 1});
        }
    n_faces = (int)face.size();
    // Parameter block: for each affine map, W [out][in] then b [out].
    int off = 0;
    for (int l = 0; l <= L; ++l) {
      int o = (l == L) ? dout : W;
      int i = (l == 0) ? din : W;
      nout.push_back(o); nin.push_back(i);
      woff.push_back(off); off += o * i;
      boff.push_back(off); off += o;
    }
    n_params = off;
  }
  bool face_is_time(int f) const { return unst && face[f][2] == ds; }
};

// ------------------------------------------------------ forward (jets) ---
// The network carries, per neuron, the value and its derivatives needed by
// the residual (Eqs. (7)-(10)): channel 0 = value, channels 1..d_in = first
// derivatives along each input (space then time), channel LAP = spatial
// Laplacian.  With jets == false only channel 0 is carried (plain value).
//
// Activation derivatives s1, s2, s3 of sigma: tanh (a = tanh z,
// s1 = 1 - a^2, s2 = -2 a s1, s3 = -2 s1 (1 - 3 a^2)) or sin (s1 = cos z,
// s2 = -sin z, s3 = -cos z; the cylinder cases of Table B1).
// Chain rule per neuron:  d_q a = s1 d_q z;
//   lap a = s2 * sum_{spatial q} (d_q z)^2 + s1 * lap z.

template <class T>
void activate(const Geo& g, int nc, const T* Z, T* A) {
  const bool sn = g.cfg.activation == 1;
  for (int k = 0; k < g.W; ++k) {
    const T* z = Z + (size_t)k * nc;
    T* a_ = A + (size_t)k * nc;
    // sigma and its first two derivatives: tanh (s1 = 1 - a^2, s2 = -2 a s1)
    // or sin (s1 = cos z, s2 = -sin z)
    T a = sn ? std::sin(z[0]) : std::tanh(z[0]);
    a_[0] = a;
    if (nc == 1) continue;
    T s1 = sn ? std::cos(z[0]) : T(1.0 - a * a);
    T s2 = sn ? T(-a) : T(-2.0 * a * s1);
    T S = 0.0;
    for (int q = 0; q < g.ds; ++q) S += z[1 + q] * z[1 + q];
    for (int q = 0; q < g.din; ++q) a_[1 + q] = s1 * z[1 + q];
    a_[g.LAP] = s2 * S + s1 * z[g.LAP];
  }
}

// Forward through net `net` at raw input x.  Stores the pre-activations of
// the L hidden layers in Z ([L][W][nc]) and the outputs in Y ([d_out][nc]).
template <class T, class X>
void forward(const Geo& g, int net, const T* th, const X* x, bool jets, T* Z, T* Y) {
  const int nc = jets ? g.C : 1;
  X xh[4];
  double s[4];
  for (int q = 0; q < g.din; ++q) {
    double c = 0.5 * (g.blo[net][q] + g.bhi[net][q]);
    s[q] = 2.0 / (g.bhi[net][q] - g.blo[net][q]);
    xh[q] = (x[q] - c) * s[q];
  }
  const T* W0 = th + g.woff[0];
  const T* b0 = th + g.boff[0];
  for (int i = 0; i < g.W; ++i) {
    T* z = Z + (size_t)i * nc;
    T v = b0[i];
    for (int q = 0; q < g.din; ++q) v += W0[i * g.din + q] * xh[q];
    z[0] = v;
    if (!jets) continue;
    for (int q = 0; q < g.din; ++q) z[1 + q] = W0[i * g.din + q] * s[q];
    z[g.LAP] = 0.0;
  }
  std::vector<T> A((size_t)g.W * nc);
  for (int l = 1; l <= g.L; ++l) {
    activate(g, nc, Z + (size_t)(l - 1) * g.W * nc, A.data());
    T* out = (l < g.L) ? Z + (size_t)l * g.W * nc : Y;
    const T* Wl = th + g.woff[l];
    const T* bl = th + g.boff[l];
    for (int i = 0; i < g.nout[l]; ++i)
      for (int ch = 0; ch < nc; ++ch) {
        T acc = (ch == 0) ? bl[i] : T(0.0);
        for (int k = 0; k < g.W; ++k) acc += Wl[i * g.W + k] * A[(size_t)k * nc + ch];
        out[(size_t)i * nc + ch] = acc;
      }
  }
}

// Navier-Stokes residuals, Eqs. (7)-(10) with 1/Re = nu; the 2D form drops
// the w and z terms, a steady problem drops the time derivative.
// Y holds [d_out][C] jets, pressure is the last output.
template <class T>
void residual(const Geo& g, const T* Y, T* r) {
  const int C = g.C, P = g.ds;
  for (int j = 0; j < g.ds; ++j) {
    T v = 0.0;
    if (g.unst) v += Y[j * C + 1 + g.ds];
    for (int i = 0; i < g.ds; ++i) v += Y[i * C] * Y[j * C + 1 + i];
    v += Y[P * C + 1 + j];
    v -= g.cfg.nu * Y[j * C + g.LAP];
    r[j] = v;
  }
  T div = 0.0;
  for (int i = 0; i < g.ds; ++i) div += Y[i * C + 1 + i];
  r[g.ds] = div;
}

// Adjoint of `residual`: accumulate d(sum_j rb_j r_j)/dY into Yb.
void residual_adjoint(const Geo& g, const double* Y, const double* rb, double* Yb) {
  const int C = g.C, P = g.ds;
  for (int j = 0; j < g.ds; ++j) {
    if (g.unst) Yb[j * C + 1 + g.ds] += rb[j];
    for (int i = 0; i < g.ds; ++i) {
      Yb[i * C] += rb[j] * Y[j * C + 1 + i];
      Yb[j * C + 1 + i] += rb[j] * Y[i * C];
    }
    Yb[P * C + 1 + j] += rb[j];
    Yb[j * C + g.LAP] += -g.cfg.nu * rb[j];
  }
  for (int i = 0; i < g.ds; ++i) Yb[i * C + 1 + i] += rb[g.ds];
}

// Adjoint of `activate` for one neuron: from the adjoints Ab of the
// activation jet to the adjoints Zb of the pre-activation jet.
void activate_adjoint(const Geo& g, int nc, const double* z, const double* Ab, double* Zb) {
  // s1, s2, s3: first three derivatives of sigma at z
  double s1, s2, s3;
  if (g.cfg.activation == 1) {
    s1 = std::cos(z[0]);
    s2 = -std::sin(z[0]);
    s3 = -s1;
  } else {
    double a = std::tanh(z[0]);
    s1 = 1.0 - a * a;
    s2 = -2.0 * a * s1;
    s3 = -2.0 * s1 * (1.0 - 3.0 * a * a);
  }
  if (nc == 1) { Zb[0] = Ab[0] * s1; return; }
  double S = 0.0;
  for (int q = 0; q < g.ds; ++q) S += z[1 + q] * z[1 + q];
  Zb[g.LAP] = Ab[g.LAP] * s1;
  double v = Ab[0] * s1 + Ab[g.LAP] * (s3 * S + s2 * z[g.LAP]);
  for (int q = 0; q < g.din; ++q) {
    double zq = (q < g.ds) ? 2.0 * Ab[g.LAP] * s2 * z[1 + q] : 0.0;
    Zb[1 + q] = Ab[1 + q] * s1 + zq;
    v += Ab[1 + q] * s2 * z[1 + q];
  }
  Zb[0] = v;
}

// Reverse pass of `forward`: given the output adjoint Yb ([d_out][nc]),
// accumulate d(sum Yb . Y)/dtheta into grad (same layout as theta).
void backward(const Geo& g, int net, const double* th, const double* x, bool jets,
              const double* Z, const double* Yb, double* grad) {
  const int nc = jets ? g.C : 1;
  std::vector<double> cur(Yb, Yb + (size_t)g.dout * nc), A((size_t)g.W * nc),
      Ab((size_t)g.W * nc), nxt((size_t)g.W * nc);
  for (int l = g.L; l >= 1; --l) {
    const double* Zp = Z + (size_t)(l - 1) * g.W * nc;
    activate(g, nc, Zp, A.data());
    const double* Wl = th + g.woff[l];
    double* dW = grad + g.woff[l];
    double* db = grad + g.boff[l];
    for (int i = 0; i < g.nout[l]; ++i) {
      db[i] += cur[(size_t)i * nc];
      for (int k = 0; k < g.W; ++k) {
        double s = 0.0;
        for (int ch = 0; ch < nc; ++ch) s += cur[(size_t)i * nc + ch] * A[(size_t)k * nc + ch];
        dW[i * g.W + k] += s;
      }
    }
    for (int k = 0; k < g.W; ++k)
      for (int ch = 0; ch < nc; ++ch) {
        double s = 0.0;
        for (int i = 0; i < g.nout[l]; ++i) s += Wl[i * g.W + k] * cur[(size_t)i * nc + ch];
        Ab[(size_t)k * nc + ch] = s;
      }
    for (int k = 0; k < g.W; ++k)
      activate_adjoint(g, nc, Zp + (size_t)k * nc, Ab.data() + (size_t)k * nc, nxt.data() + (size_t)k * nc);
    cur = nxt;
  }
  // First affine map: z = W0 xh + b0, d_q z = s_q W0[:, q], lap z = 0.
  double xh[4], s[4];
  for (int q = 0; q < g.din; ++q) {
    double c = 0.5 * (g.blo[net][q] + g.bhi[net][q]);
    s[q] = 2.0 / (g.bhi[net][q] - g.blo[net][q]);
    xh[q] = (x[q] - c) * s[q];
  }
  double* dW0 = grad + g.woff[0];
  double* db0 = grad + g.boff[0];
  for (int i = 0; i < g.W; ++i) {
    db0[i] += cur[(size_t)i * nc];
    for (int q = 0; q < g.din; ++q) {
      double v = cur[(size_t)i * nc] * xh[q];
      if (jets) v += cur[(size_t)i * nc + 1 + q] * s[q];
      dW0[i * g.din + q] += v;
    }
  }
}

// --------------------------------------------------------------- problem ---
struct Prob {
  const Geo& g;
  const ora_problem& p;
  std::vector<int64_t> res_off, obs_off, face_off;
  Prob(const Geo& g_, const ora_problem& p_) : g(g_), p(p_) {
    int64_t o = 0;
    for (int k = 0; k < g.n_nets; ++k) { res_off.push_back(o); o += p.res_counts ? p.res_counts[k] : 0; }
    res_off.push_back(o);
    o = 0;
    for (int k = 0; k < g.n_nets; ++k) { obs_off.push_back(o); o += p.obs_counts ? p.obs_counts[k] : 0; }
    obs_off.push_back(o);
    o = 0;
    for (int f = 0; f < g.n_faces; ++f) { face_off.push_back(o); o += p.face_counts ? p.face_counts[f] : 0; }
    face_off.push_back(o);
    o = 0;
    for (int k = 0; k < g.n_nets; ++k) { ghost_off.push_back(o); o += p.ghost_counts ? p.ghost_counts[k] : 0; }
    ghost_off.push_back(o);
  }
  bool ghost_mode() const { return p.ghost_counts != nullptr; }
  void ghost_x(int64_t i, double* x) const { for (int q = 0; q < g.din; ++q) x[q] = p.ghost_pts[i * g.din + q]; }
  std::vector<int64_t> ghost_off;
  void res_x(int64_t i, double* x) const { for (int q = 0; q < g.din; ++q) x[q] = p.res_pts[i * g.din + q]; }
  void obs_x(int64_t i, double* x) const { for (int q = 0; q < g.din; ++q) x[q] = p.obs_pts[i * g.din + q]; }
  void face_x(int64_t i, double* x) const { for (int q = 0; q < g.din; ++q) x[q] = p.face_pts[i * g.din + q]; }
  int64_t n_gh(int net) const {
    if (ghost_mode()) return ghost_off[net + 1] - ghost_off[net];
    int64_t n = 0;
    for (auto& fs : g.net_faces[net]) n += face_off[fs.first + 1] - face_off[fs.first];
    return n;
  }
};

// Neighbour messages at the current parameters (Algorithm 1, exchange step):
// val[pt][side][d_out] = net_side(x_pt); anc[pt][side] = p_side(x_anc, t_pt)
// for a master side (0 otherwise).
struct Nbr {
  std::vector<double> val, anc;
  // with the interface terms: the other side's residual [pt][2][d_s + 1]
  // and first derivatives [pt][2][d_out][d_in]
  std::vector<double> res, grd;
  // ghost mode: per ghost point, the owner net and its (u, p) and anchor p
  // (and residual [pt][d_s + 1] and first derivatives [pt][d_out][d_in])
  std::vector<int> owner;
  std::vector<double> gval, ganc, gres, ggrd;
};

constexpr int NLOSS = 8;   // loss record: obs, PDE, gh_u, gh_p space, gh_p time, total, gh_r, gh_c1

bool iface_jets(const Geo& g) { return g.cfg.lam_gh_r != 0.0 || g.cfg.lam_gh_c1 != 0.0; }

// Residual and first derivatives of net `net` at x from its jets.
void point_jets(const Geo& g, int net, const double* th, const double* x, double* r, double* grd) {
  std::vector<double> Z((size_t)g.L * g.W * g.C), Y((size_t)g.dout * g.C);
  forward(g, net, th, x, true, Z.data(), Y.data());
  residual(g, Y.data(), r);
  for (int c = 0; c < g.dout; ++c)
    for (int q = 0; q < g.din; ++q) grd[c * g.din + q] = Y[c * g.C + 1 + q];
}

// Net whose cell holds x (float32 rule), -1 outside the domain.
int route_fp32(const Geo& g, const double* x) {
  int net = 0;
  for (int a = 0; a < g.din; ++a) {
    int k = cell_fp32(g.cfg, a, (float)x[a]);
    if (k < 0) return -1;
    net += k * g.stride[a];
  }
  return net;
}

// The anchor's coordinates are taken at float32 precision, the precision of
// every point the method is given, so a query point placed on x_anc hits it
// exactly.
void anchor_point(const Geo& g, const double* x, double* xa) {
  for (int q = 0; q < g.ds; ++q) xa[q] = (double)(float)g.cfg.anchor[q];
  if (g.unst) xa[g.ds] = x[g.ds];
}

template <class T>
T value_p(const Geo& g, int net, const T* th, const double* x) {
  std::vector<T> Z((size_t)g.L * g.W), Y(g.dout);
  forward(g, net, th, x, false, Z.data(), Y.data());
  return Y[g.ds];
}

// Only faces touching a net flagged in `need` are evaluated (all when null);
// the others keep zeros and are never read by those nets' losses.
Nbr exchange(const Prob& pb, const double* th_all, const std::vector<char>* need = nullptr) {
  const Geo& g = pb.g;
  Nbr nb;
  if (pb.ghost_mode()) {
    // each ghost point of net A is evaluated by the net B whose cell holds it
    const int64_t n = pb.ghost_off.back();
    nb.owner.assign(n, -1);
    nb.gval.assign((size_t)n * g.dout, 0.0);
    nb.ganc.assign(n, 0.0);
    if (iface_jets(g)) {
      nb.gres.assign((size_t)n * (g.ds + 1), 0.0);
      nb.ggrd.assign((size_t)n * g.dout * g.din, 0.0);
    }
    std::vector<double> Zg((size_t)g.L * g.W), Yg(g.dout);
    for (int A = 0; A < g.n_nets; ++A) {
      if (need && !(*need)[A]) continue;
      for (int64_t i = pb.ghost_off[A]; i < pb.ghost_off[A + 1]; ++i) {
        double x[4], xa[4];
        pb.ghost_x(i, x);
        const int B = route_fp32(g, x);
        nb.owner[i] = B;
        if (B < 0) continue;
        const double* th = th_all + (size_t)B * g.n_params;
        forward(g, B, th, x, false, Zg.data(), Yg.data());
        for (int j = 0; j < g.dout; ++j) nb.gval[(size_t)i * g.dout + j] = Yg[j];
        if (iface_jets(g))
          point_jets(g, B, th, x, &nb.gres[(size_t)i * (g.ds + 1)], &nb.ggrd[(size_t)i * g.dout * g.din]);
        if (g.master[B]) {
          anchor_point(g, x, xa);
          nb.ganc[i] = value_p(g, B, th, xa);
        }
      }
    }
    return nb;
  }
  int64_t nf = pb.face_off.back();
  nb.val.assign((size_t)nf * 2 * g.dout, 0.0);
  nb.anc.assign((size_t)nf * 2, 0.0);
  if (iface_jets(g)) {
    nb.res.assign((size_t)nf * 2 * (g.ds + 1), 0.0);
    nb.grd.assign((size_t)nf * 2 * g.dout * g.din, 0.0);
  }
  std::vector<double> Z((size_t)g.L * g.W), Y(g.dout);
  for (int f = 0; f < g.n_faces; ++f) {
    if (need && !(*need)[g.face[f][0]] && !(*need)[g.face[f][1]]) continue;
    for (int64_t i = pb.face_off[f]; i < pb.face_off[f + 1]; ++i) {
      double x[4], xa[4];
      pb.face_x(i, x);
      for (int side = 0; side < 2; ++side) {
        int net = g.face[f][side];
        const double* th = th_all + (size_t)net * g.n_params;
        forward(g, net, th, x, false, Z.data(), Y.data());
        for (int j = 0; j < g.dout; ++j) nb.val[((size_t)i * 2 + side) * g.dout + j] = Y[j];
        if (iface_jets(g))
          point_jets(g, net, th, x, &nb.res[((size_t)i * 2 + side) * (g.ds + 1)],
                     &nb.grd[((size_t)i * 2 + side) * g.dout * g.din]);
        if (g.master[net]) {  // Eq. (15): master sends p~ = p(x,t) - p(x_anc,t)
          anchor_point(g, x, xa);
          nb.anc[(size_t)i * 2 + side] = value_p(g, net, th, xa);
        }
      }
    }
  }
  return nb;
}

// Target the own side `side` of face point i is pulled towards: the other
// side's velocity and (anchor-normalised if the other side is a master)
// pressure, held constant.
void ghost_target(const Prob& pb, const Nbr& nb, int f, int64_t i, int side, double* U, double* P) {
  const Geo& g = pb.g;
  int other = 1 - side;
  int nb_net = g.face[f][other];
  const double* v = &nb.val[((size_t)i * 2 + other) * g.dout];
  for (int c = 0; c < g.ds; ++c) U[c] = v[c];
  *P = v[g.ds] - (g.master[nb_net] ? nb.anc[(size_t)i * 2 + other] : 0.0);
}

double lam_space(const Geo& g, int net) { return g.master[net] ? 0.0 : g.cfg.lam_gh_p_space; }

// Volumetric ghost point i of net A: the owner B's velocity and (anchor-
// normalised if B is a master) pressure; the pressure term is temporal when
// A and B share their spatial cell (a purely temporal neighbour).
void ghost_target_vol(const Prob& pb, const Nbr& nb, int A, int64_t i, double* U, double* P, bool* is_time) {
  const Geo& g = pb.g;
  const int B = nb.owner[i];
  const double* v = &nb.gval[(size_t)i * g.dout];
  for (int c = 0; c < g.ds; ++c) U[c] = v[c];
  *P = v[g.ds] - (g.master[B] ? nb.ganc[i] : 0.0);
  bool same_space = true;
  for (int a = 0; a < g.ds; ++a) same_space = same_space && g.cell[A][a] == g.cell[B][a];
  *is_time = g.unst && same_space;
}

// The other side's residual and first derivatives at ghost point i (face
// mode: face f, own side `side`; ghost mode: the owner of point i).
void jet_targets(const Prob& pb, const Nbr& nb, bool ghost, int f_unused, int64_t i, int side, const double** rB,
                 const double** gB) {
  const Geo& g = pb.g;
  (void)f_unused;
  if (ghost) {
    *rB = &nb.gres[(size_t)i * (g.ds + 1)];
    *gB = &nb.ggrd[(size_t)i * g.dout * g.din];
  } else {
    const int other = 1 - side;
    *rB = &nb.res[((size_t)i * 2 + other) * (g.ds + 1)];
    *gB = &nb.grd[((size_t)i * 2 + other) * g.dout * g.din];
  }
}

// Loss terms of net A at parameters thA (T = double or complex for the
// complex-step pins): out = {L_obs, L_PDE, L_gh_u, L_gh_p^space,
// L_gh_p^time, L_total, L_gh_r, L_gh_c1}.  Eq. (3), Eq. (5), Eqs. (13)-(14),
// Eq. (16), and the optional interface terms of the Remark in Sec. 2.2.
template <class T>
void net_loss(const Prob& pb, const Nbr& nb, int A, const T* thA, T* out) {
  const Geo& g = pb.g;
  T lobs = 0.0, lpde = 0.0, lgu = 0.0, lsp = 0.0, ltm = 0.0;
  std::vector<T> Z((size_t)g.L * g.W * g.C), Y((size_t)g.dout * g.C), r(g.ds + 1);
  std::vector<T> Zv((size_t)g.L * g.W), Yv(g.dout);
  int64_t npde = pb.res_off[A + 1] - pb.res_off[A];
  for (int64_t i = pb.res_off[A]; i < pb.res_off[A + 1]; ++i) {
    double x[4];
    pb.res_x(i, x);
    forward(g, A, thA, x, true, Z.data(), Y.data());
    residual(g, Y.data(), r.data());
    for (int j = 0; j <= g.ds; ++j) lpde += r[j] * r[j];
  }
  int64_t nobs = pb.obs_off[A + 1] - pb.obs_off[A];
  for (int64_t i = pb.obs_off[A]; i < pb.obs_off[A + 1]; ++i) {
    double x[4];
    pb.obs_x(i, x);
    forward(g, A, thA, x, false, Zv.data(), Yv.data());
    for (int c = 0; c < g.ds; ++c) {
      T e = Yv[c] - (double)pb.p.obs_vals[i * g.ds + c];
      lobs += g.cfg.comp_w[c] * e * e;
    }
  }
  int64_t ngh = pb.n_gh(A);
  T lr = 0.0, lc1 = 0.0;
  std::vector<T> rj(g.ds + 1);
  // one ghost point: C0 terms (Eqs. (13)-(14)) and, when enabled, residual
  // and C1 matching against the other side's jets
  auto ghost_point = [&](const double* x, const double* U, double P, bool tm, const double* rB, const double* gB) {
    const bool jets = iface_jets(g);
    if (jets) forward(g, A, thA, x, true, Z.data(), Y.data());
    else forward(g, A, thA, x, false, Zv.data(), Yv.data());
    const int st = jets ? g.C : 1;
    const T* Yc = jets ? Y.data() : Yv.data();
    for (int c = 0; c < g.ds; ++c) {
      T e = Yc[c * st] - U[c];
      lgu += g.cfg.comp_w[c] * e * e;
    }
    T ep = Yc[g.ds * st] - P;
    if (tm) ltm += ep * ep; else lsp += ep * ep;
    if (jets) {
      residual(g, Y.data(), rj.data());
      for (int j = 0; j <= g.ds; ++j) {
        T d = rj[j] - rB[j];
        lr += d * d;
      }
      for (int c = 0; c < g.dout; ++c)
        for (int q = 0; q < g.din; ++q) {
          T d = Y[c * g.C + 1 + q] - gB[c * g.din + q];
          lc1 += d * d;
        }
    }
  };
  for (auto& fs : g.net_faces[A]) {
    if (pb.ghost_mode()) break;
    int f = fs.first, side = fs.second;
    for (int64_t i = pb.face_off[f]; i < pb.face_off[f + 1]; ++i) {
      double x[4], U[3], P;
      const double *rB = nullptr, *gB = nullptr;
      pb.face_x(i, x);
      ghost_target(pb, nb, f, i, side, U, &P);
      if (iface_jets(g)) jet_targets(pb, nb, false, f, i, side, &rB, &gB);
      ghost_point(x, U, P, g.face_is_time(f), rB, gB);
    }
  }
  if (pb.ghost_mode())
    for (int64_t i = pb.ghost_off[A]; i < pb.ghost_off[A + 1]; ++i) {
      double x[4], U[3], P;
      bool tm;
      const double *rB = nullptr, *gB = nullptr;
      pb.ghost_x(i, x);
      ghost_target_vol(pb, nb, A, i, U, &P, &tm);
      if (iface_jets(g)) jet_targets(pb, nb, true, 0, i, 0, &rB, &gB);
      ghost_point(x, U, P, tm, rB, gB);
    }
  out[0] = nobs ? lobs / (double)nobs : T(0.0);
  out[1] = npde ? lpde / (double)npde : T(0.0);
  out[2] = ngh ? lgu / (double)ngh : T(0.0);
  out[3] = ngh ? lsp / (double)ngh : T(0.0);
  out[4] = ngh ? ltm / (double)ngh : T(0.0);
  out[6] = ngh ? lr / (double)ngh : T(0.0);
  out[7] = ngh ? lc1 / (double)ngh : T(0.0);
  out[5] = g.cfg.lam_obs * out[0] + g.cfg.lam_pde * out[1] + g.cfg.lam_gh_u * out[2] +
           lam_space(g, A) * out[3] + g.cfg.lam_gh_p_time * out[4] + g.cfg.lam_gh_r * out[6] +
           g.cfg.lam_gh_c1 * out[7];
}

// Hand-written gradient of L_A with respect to theta_A (neighbour values are
// constants, so the total gradient is block-diagonal over nets).  Points are
// split statically over g_threads threads; per-thread sums are added in
// thread order, so the result is deterministic for a fixed thread count.
void net_grad(const Prob& pb, const Nbr& nb, int A, const double* thA, double* grad, double* loss) {
  const Geo& g = pb.g;
  int64_t npde = pb.res_off[A + 1] - pb.res_off[A];
  int64_t nobs = pb.obs_off[A + 1] - pb.obs_off[A];
  int64_t ngh = pb.n_gh(A);
  // Flat list of work: residual points, obs points, then (face, side, point).
  struct Item { int kind; int f; int side; int64_t i; };
  std::vector<Item> items;
  for (int64_t i = pb.res_off[A]; i < pb.res_off[A + 1]; ++i) items.push_back({0, 0, 0, i});
  for (int64_t i = pb.obs_off[A]; i < pb.obs_off[A + 1]; ++i) items.push_back({1, 0, 0, i});
  if (pb.ghost_mode()) {
    for (int64_t i = pb.ghost_off[A]; i < pb.ghost_off[A + 1]; ++i) items.push_back({3, 0, 0, i});
  } else {
    for (auto& fs : g.net_faces[A])
      for (int64_t i = pb.face_off[fs.first]; i < pb.face_off[fs.first + 1]; ++i)
        items.push_back({2, fs.first, fs.second, i});
  }
  int T = std::max(1, g_threads);
  std::vector<std::vector<double>> gbuf(T, std::vector<double>(g.n_params, 0.0));
  std::vector<std::array<double, 7>> lbuf(T, {0, 0, 0, 0, 0, 0, 0});
  auto work = [&](int t) {
    size_t n = items.size();
    size_t b = n * t / T, e = n * (t + 1) / T;
    std::vector<double> Z((size_t)g.L * g.W * g.C), Y((size_t)g.dout * g.C), Yb((size_t)g.dout * g.C);
    double r[4], rb[4];
    for (size_t it = b; it < e; ++it) {
      const Item& w = items[it];
      double x[4];
      std::fill(Yb.begin(), Yb.end(), 0.0);
      if (w.kind == 0) {
        pb.res_x(w.i, x);
        forward(g, A, thA, x, true, Z.data(), Y.data());
        residual(g, Y.data(), r);
        for (int j = 0; j <= g.ds; ++j) {
          lbuf[t][1] += r[j] * r[j];
          rb[j] = 2.0 * g.cfg.lam_pde * r[j] / (double)npde;
        }
        residual_adjoint(g, Y.data(), rb, Yb.data());
        backward(g, A, thA, x, true, Z.data(), Yb.data(), gbuf[t].data());
      } else if (w.kind == 1) {
        pb.obs_x(w.i, x);
        forward(g, A, thA, x, false, Z.data(), Y.data());
        for (int c = 0; c < g.ds; ++c) {
          double e_ = Y[c] - (double)pb.p.obs_vals[w.i * g.ds + c];
          lbuf[t][0] += g.cfg.comp_w[c] * e_ * e_;
          Yb[c] = 2.0 * g.cfg.lam_obs * g.cfg.comp_w[c] * e_ / (double)nobs;
        }
        backward(g, A, thA, x, false, Z.data(), Yb.data(), gbuf[t].data());
      } else {
        double U[3], P;
        bool tm;
        const double *rB = nullptr, *gB = nullptr;
        if (w.kind == 2) {
          pb.face_x(w.i, x);
          ghost_target(pb, nb, w.f, w.i, w.side, U, &P);
          tm = g.face_is_time(w.f);
        } else {
          pb.ghost_x(w.i, x);
          ghost_target_vol(pb, nb, A, w.i, U, &P, &tm);
        }
        const bool jets = iface_jets(g);
        if (jets) jet_targets(pb, nb, w.kind == 3, w.f, w.i, w.side, &rB, &gB);
        forward(g, A, thA, x, jets, Z.data(), Y.data());
        const int st = jets ? g.C : 1;   // value channel stride
        for (int c = 0; c < g.ds; ++c) {
          double e_ = Y[c * st] - U[c];
          lbuf[t][2] += g.cfg.comp_w[c] * e_ * e_;
          Yb[c * st] = 2.0 * g.cfg.lam_gh_u * g.cfg.comp_w[c] * e_ / (double)ngh;
        }
        double ep = Y[g.ds * st] - P;
        lbuf[t][tm ? 4 : 3] += ep * ep;
        double lam = tm ? g.cfg.lam_gh_p_time : lam_space(g, A);
        Yb[g.ds * st] = 2.0 * lam * ep / (double)ngh;
        if (jets) {
          // residual matching: d/dY of lam_r / N_gh sum_j (r_j - rB_j)^2
          residual(g, Y.data(), r);
          for (int j = 0; j <= g.ds; ++j) {
            const double d = r[j] - rB[j];
            lbuf[t][5] += d * d;
            rb[j] = 2.0 * g.cfg.lam_gh_r * d / (double)ngh;
          }
          residual_adjoint(g, Y.data(), rb, Yb.data());
          // C1 matching on every first derivative of every output
          for (int c = 0; c < g.dout; ++c)
            for (int q = 0; q < g.din; ++q) {
              const double d = Y[c * g.C + 1 + q] - gB[c * g.din + q];
              lbuf[t][6] += d * d;
              Yb[c * g.C + 1 + q] += 2.0 * g.cfg.lam_gh_c1 * d / (double)ngh;
            }
        }
        backward(g, A, thA, x, jets, Z.data(), Yb.data(), gbuf[t].data());
      }
    }
  };
  if (T == 1) work(0);
  else {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  std::fill(grad, grad + g.n_params, 0.0);
  double l[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    for (int j = 0; j < g.n_params; ++j) grad[j] += gbuf[t][j];
    for (int q = 0; q < 7; ++q) l[q] += lbuf[t][q];
  }
  if (loss) {
    loss[0] = nobs ? l[0] / nobs : 0.0;
    loss[1] = npde ? l[1] / npde : 0.0;
    loss[2] = ngh ? l[2] / ngh : 0.0;
    loss[3] = ngh ? l[3] / ngh : 0.0;
    loss[4] = ngh ? l[4] / ngh : 0.0;
    loss[6] = ngh ? l[5] / ngh : 0.0;
    loss[7] = ngh ? l[6] / ngh : 0.0;
    loss[5] = g.cfg.lam_obs * loss[0] + g.cfg.lam_pde * loss[1] + g.cfg.lam_gh_u * loss[2] +
              lam_space(g, A) * loss[3] + g.cfg.lam_gh_p_time * loss[4] + g.cfg.lam_gh_r * loss[6] +
              g.cfg.lam_gh_c1 * loss[7];
  }
}

// Optional per-net clipping then Adam (PyTorch's rule, no weight decay):
// m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
// theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
void adam(const Geo& g, double* th, double* m, double* v, int64_t t, const double* grad_in) {
  const ora_config& c = g.cfg;
  std::vector<double> gr(grad_in, grad_in + (size_t)g.n_nets * g.n_params);
  if (c.clip > 0.0)
    for (int k = 0; k < g.n_nets; ++k) {
      double n2 = 0.0;
      for (int j = 0; j < g.n_params; ++j) n2 += gr[(size_t)k * g.n_params + j] * gr[(size_t)k * g.n_params + j];
      double coef = c.clip / (std::sqrt(n2) + 1e-6);
      if (coef < 1.0)
        for (int j = 0; j < g.n_params; ++j) gr[(size_t)k * g.n_params + j] *= coef;
    }
  double bc1 = 1.0 - std::pow(c.beta1, (double)t);
  double bc2 = 1.0 - std::pow(c.beta2, (double)t);
  double lr = c.lr;
  if (c.lr_decay_interval > 0) lr *= std::pow(c.lr_decay_factor, (double)((t - 1) / c.lr_decay_interval));
  for (size_t j = 0; j < gr.size(); ++j) {
    m[j] = c.beta1 * m[j] + (1.0 - c.beta1) * gr[j];
    v[j] = c.beta2 * v[j] + (1.0 - c.beta2) * gr[j] * gr[j];
    double mh = m[j] / bc1, vh = v[j] / bc2;
    th[j] -= lr * mh / (std::sqrt(vh) + c.eps);
  }
}

}  // namespace

// ------------------------------------------------- collocation sampler ---
// Uniform collocation points in each net's interior cell for step t, from
// counter-based SplitMix64 streams (Steele, Lea, Flood 2014): the generator
// seeded with S yields mix(S + n * gamma) as its n-th output (n = 1, 2, ...),
// mix being its output function.  Step stream S_t = output t + 1 of the seed;
// net stream S_{t,k} = output k + 1 of S_t; axis d of point i takes output
// i * d_in + d + 1 of S_{t,k}, its top 24 bits giving u in [0, 1); the point
// is lo + u (hi - lo) in double, rounded to float32.  (A sampling scheme the
// paper leaves open; it trains on fixed point sets, Sec. 3.)
static uint64_t splitmix64_output(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}
static uint64_t splitmix64_nth(uint64_t seed, uint64_t n) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ull;
  return splitmix64_output(seed + n * gamma);
}

// ================================================================ C API ===
extern "C" {

void ora_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

// Layout: counts, per-net master flag and box, faces (lo, hi, axis, is_time).
int ora_layout(const ora_config* c, int* n_nets, int* n_faces, int* n_params,
               int* master, double* box_lo, double* box_hi, int* faces) {
  Geo g(*c);
  if (n_nets) *n_nets = g.n_nets;
  if (n_faces) *n_faces = g.n_faces;
  if (n_params) *n_params = g.n_params;
  for (int k = 0; master && k < g.n_nets; ++k) master[k] = g.master[k];
  for (int k = 0; box_lo && k < g.n_nets; ++k)
    for (int q = 0; q < 4; ++q) { box_lo[k * 4 + q] = g.blo[k][q]; box_hi[k * 4 + q] = g.bhi[k][q]; }
  for (int f = 0; faces && f < g.n_faces; ++f) {
    faces[f * 4 + 0] = g.face[f][0]; faces[f * 4 + 1] = g.face[f][1];
    faces[f * 4 + 2] = g.face[f][2]; faces[f * 4 + 3] = g.face_is_time(f) ? 1 : 0;
  }
  return 0;
}

// n-th output of the SplitMix64 generator seeded with `seed` (tests).
uint64_t ora_splitmix64_nth(uint64_t seed, uint64_t n) { return splitmix64_nth(seed, n); }

// Collocation points of step t: counts[k] points of net k, concatenated in
// net order, out [sum counts][d_in] float32.
int ora_sample(const ora_config* c, uint64_t seed, int64_t t, const int64_t* counts, float* out) {
  Geo g(*c);
  int64_t row = 0;
  const uint64_t s_t = splitmix64_nth(seed, (uint64_t)t + 1);
  for (int k = 0; k < g.n_nets; ++k) {
    const uint64_t s_tk = splitmix64_nth(s_t, (uint64_t)k + 1);
    for (int64_t i = 0; i < counts[k]; ++i, ++row)
      for (int d = 0; d < g.din; ++d) {
        const uint64_t o = splitmix64_nth(s_tk, (uint64_t)(i * g.din + d) + 1);
        const double u = (double)(o >> 40) / 16777216.0;
        const double x = g.blo[k][d] + u * (g.bhi[k][d] - g.blo[k][d]);
        out[row * g.din + d] = (float)x;
      }
  }
  return 0;
}

// Jets (jets = 1: out [n][d_out][C]) or values (jets = 0: out [n][d_out]) of
// net `net` with parameters th_net at double points x [n][d_in].
int ora_forward(const ora_config* c, int net, const double* th_net, const double* x, int64_t n,
                int jets, double* out) {
  Geo g(*c);
  int nc = jets ? g.C : 1;
  std::vector<double> Z((size_t)g.L * g.W * nc), Y((size_t)g.dout * nc);
  for (int64_t i = 0; i < n; ++i) {
    forward(g, net, th_net, x + i * g.din, jets != 0, Z.data(), Y.data());
    std::copy(Y.begin(), Y.end(), out + (size_t)i * g.dout * nc);
  }
  return 0;
}

// Complex-step variant: parameters th_re + i th_im, inputs x_re + i x_im.
int ora_forward_complex(const ora_config* c, int net, const double* th_re, const double* th_im,
                        const double* x_re, const double* x_im, int64_t n, int jets,
                        double* out_re, double* out_im) {
  Geo g(*c);
  int nc = jets ? g.C : 1;
  std::vector<cplx> th(g.n_params);
  for (int j = 0; j < g.n_params; ++j) th[j] = cplx(th_re[j], th_im ? th_im[j] : 0.0);
  std::vector<cplx> Z((size_t)g.L * g.W * nc), Y((size_t)g.dout * nc);
  for (int64_t i = 0; i < n; ++i) {
    cplx x[4];
    for (int q = 0; q < g.din; ++q) x[q] = cplx(x_re[i * g.din + q], x_im ? x_im[i * g.din + q] : 0.0);
    forward(g, net, th.data(), x, jets != 0, Z.data(), Y.data());
    for (size_t j = 0; j < Y.size(); ++j) {
      out_re[(size_t)i * Y.size() + j] = Y[j].real();
      out_im[(size_t)i * Y.size() + j] = Y[j].imag();
    }
  }
  return 0;
}

// Residuals r [n][d_space+1] from output jets Y [n][d_out][C].
int ora_residual(const ora_config* c, const double* Y, int64_t n, double* r) {
  Geo g(*c);
  for (int64_t i = 0; i < n; ++i) residual(g, Y + (size_t)i * g.dout * g.C, r + (size_t)i * (g.ds + 1));
  return 0;
}

// Vector-Jacobian product of the forward pass at one point:
// grad = d(sum Yb . Y)/dtheta for net `net`.
int ora_forward_vjp(const ora_config* c, int net, const double* th_net, const double* x, int jets,
                    const double* Yb, double* grad) {
  Geo g(*c);
  int nc = jets ? g.C : 1;
  std::vector<double> Z((size_t)g.L * g.W * nc), Y((size_t)g.dout * nc);
  forward(g, net, th_net, x, jets != 0, Z.data(), Y.data());
  std::fill(grad, grad + g.n_params, 0.0);
  backward(g, net, th_net, x, jets != 0, Z.data(), Yb, grad);
  return 0;
}

// Adjoint of the residual at one point: Yb = d(sum rb . r)/dY.
int ora_residual_vjp(const ora_config* c, const double* Y, const double* rb, double* Yb) {
  Geo g(*c);
  std::fill(Yb, Yb + (size_t)g.dout * g.C, 0.0);
  residual_adjoint(g, Y, rb, Yb);
  return 0;
}

// Neighbour messages: val [n_face_pts][2][d_out], anc [n_face_pts][2].
int ora_exchange(const ora_config* c, const ora_problem* p, const double* th, double* val, double* anc) {
  Geo g(*c);
  Prob pb(g, *p);
  Nbr nb = exchange(pb, th);
  std::copy(nb.val.begin(), nb.val.end(), val);
  std::copy(nb.anc.begin(), nb.anc.end(), anc);
  return 0;
}

// Loss record [n_nets][8] by direct evaluation (no derivatives of theta).
int ora_losses(const ora_config* c, const ora_problem* p, const double* th, double* out) {
  Geo g(*c);
  Prob pb(g, *p);
  Nbr nb = exchange(pb, th);
  for (int k = 0; k < g.n_nets; ++k) net_loss<double>(pb, nb, k, th + (size_t)k * g.n_params, out + k * NLOSS);
  return 0;
}

// Loss of net A with its own parameters thA_re + i thA_im, all neighbour
// messages computed from the real parameters th (held constant, as the
// paper's cached neighbour values).  Serves both the complex-step pins
// (thA_im = perturbation) and central differences (thA_re shifted).
// out_re/out_im [8].
int ora_net_loss_complex(const ora_config* c, const ora_problem* p, const double* th, int A,
                         const double* thA_re, const double* thA_im, double* out_re, double* out_im) {
  Geo g(*c);
  Prob pb(g, *p);
  Nbr nb = exchange(pb, th);
  std::vector<cplx> thA(g.n_params);
  for (int j = 0; j < g.n_params; ++j)
    thA[j] = cplx(thA_re ? thA_re[j] : th[(size_t)A * g.n_params + j], thA_im ? thA_im[j] : 0.0);
  cplx out[NLOSS];
  net_loss<cplx>(pb, nb, A, thA.data(), out);
  for (int q = 0; q < NLOSS; ++q) { out_re[q] = out[q].real(); out_im[q] = out[q].imag(); }
  return 0;
}

// Gradient (hand-written reverse pass) and loss record for the selected nets:
// grad [n_sel][n_params], loss [n_sel][8].
int ora_grad_nets(const ora_config* c, const ora_problem* p, const double* th, const int* nets,
                  int n_sel, double* grad, double* loss) {
  Geo g(*c);
  Prob pb(g, *p);
  std::vector<char> need(g.n_nets, 0);
  for (int s = 0; s < n_sel; ++s) need[nets[s]] = 1;
  Nbr nb = exchange(pb, th, &need);
  for (int s = 0; s < n_sel; ++s) {
    int A = nets[s];
    net_grad(pb, nb, A, th + (size_t)A * g.n_params, grad + (size_t)s * g.n_params, loss ? loss + s * NLOSS : nullptr);
  }
  return 0;
}

int ora_grad(const ora_config* c, const ora_problem* p, const double* th, double* grad, double* loss) {
  Geo g(*c);
  std::vector<int> nets(g.n_nets);
  for (int k = 0; k < g.n_nets; ++k) nets[k] = k;
  return ora_grad_nets(c, p, th, nets.data(), g.n_nets, grad, loss);
}

// Adam (with optional clipping) alone: t is incremented first.
int ora_adam(const ora_config* c, double* th, double* m, double* v, int64_t* t, const double* grad) {
  Geo g(*c);
  *t += 1;
  adam(g, th, m, v, *t, grad);
  return 0;
}

// One full training iteration of Algorithm 1 with I_comm = 1: exchange,
// losses and gradients at the current parameters, then the optimiser step.
// loss [n_nets][8] holds the pre-update losses.
int ora_step(const ora_config* c, const ora_problem* p, double* th, double* m, double* v,
             int64_t* t, double* loss) {
  Geo g(*c);
  std::vector<double> grad((size_t)g.n_nets * g.n_params);
  ora_grad(c, p, th, grad.data(), loss);
  *t += 1;
  adam(g, th, m, v, *t, grad.data());
  return 0;
}

// One iteration of Algorithm 1 with a communication interval: the neighbour
// messages are recomputed into (val, anc) when t mod I_comm == 0 (t = steps
// taken so far) and the cached ones are used otherwise; then losses,
// gradients and the optimiser step.  val [n_face_pts][2][d_out],
// anc [n_face_pts][2] persist between calls.
int ora_step_cached(const ora_config* c, const ora_problem* p, double* th, double* m, double* v, int64_t* t,
                    double* loss, double* val, double* anc) {
  Geo g(*c);
  Prob pb(g, *p);
  Nbr nb;
  const int64_t nf = pb.face_off.back();
  if (iface_jets(g) && c->comm_interval > 1) return -2;   // the cache holds values only
  if (c->comm_interval <= 1 || (*t % c->comm_interval) == 0) {
    nb = exchange(pb, th);
    std::copy(nb.val.begin(), nb.val.end(), val);
    std::copy(nb.anc.begin(), nb.anc.end(), anc);
  } else {
    nb.val.assign(val, val + (size_t)nf * 2 * g.dout);
    nb.anc.assign(anc, anc + (size_t)nf * 2);
  }
  std::vector<double> grad((size_t)g.n_nets * g.n_params);
  for (int k = 0; k < g.n_nets; ++k)
    net_grad(pb, nb, k, th + (size_t)k * g.n_params, grad.data() + (size_t)k * g.n_params, loss ? loss + k * NLOSS : nullptr);
  *t += 1;
  adam(g, th, m, v, *t, grad.data());
  return 0;
}

// Query: route each float32 point to its cell (FP32 rule), evaluate the net;
// output [n][d_out] or, with want_res, [n][d_out + d_space + 1] with the
// residuals appended.  Pressure output: p - p(x_anc, t) + p_ref in master
// cells, p + p_ref elsewhere (Eq. (18)).  Returns -1 if a point lies
// outside the domain (its output row is left untouched).
int ora_query(const ora_config* c, const double* th_all, const float* pts, int64_t n, int want_res,
              double* out, int* net_out) {
  Geo g(*c);
  int w = g.dout + (want_res ? g.ds + 1 : 0);
  std::vector<double> Z((size_t)g.L * g.W * g.C), Y((size_t)g.dout * g.C), r(g.ds + 1);
  int status = 0;
  for (int64_t i = 0; i < n; ++i) {
    int net = 0;
    bool ok = true;
    for (int a = g.din - 1; a >= 0; --a) {
      int k = cell_fp32(*c, a, pts[i * g.din + a]);
      if (k < 0) { ok = false; break; }
      net += k * g.stride[a];
    }
    if (net_out) net_out[i] = ok ? net : -1;
    if (!ok) { status = -1; continue; }
    double x[4];
    for (int q = 0; q < g.din; ++q) x[q] = pts[i * g.din + q];
    const double* th = th_all + (size_t)net * g.n_params;
    double* o = out + (size_t)i * w;
    int nc = want_res ? g.C : 1;
    forward(g, net, th, x, want_res != 0, Z.data(), Y.data());
    for (int j = 0; j < g.dout; ++j) o[j] = Y[(size_t)j * nc];
    if (g.master[net]) {
      double xa[4];
      anchor_point(g, x, xa);
      o[g.ds] = o[g.ds] - value_p(g, net, th, xa);
    }
    o[g.ds] = o[g.ds] + c->p_ref;
    if (want_res) {
      residual(g, Y.data(), r.data());
      for (int j = 0; j <= g.ds; ++j) o[g.dout + j] = r[j];
    }
  }
  return status;
}

}  // extern "C"

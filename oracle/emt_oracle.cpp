// Plain FP64 CPU oracle of the EMTP-type time loop -- TEST INFRASTRUCTURE.
//
// Only the tests, the package smoke check and the benchmark's CPU-baseline
// leg load this file's library.  It shares nothing with the CUDA path.
//
// What it computes (the four basic processes of the EMTP-type algorithm,
// CloudPSS paper Sec. III-A, with the textbook formulas of its ref. [2]):
//
//   companion conductances (trapezoidal rule)
//     R: g = 1/R        L: g = dt/(2L)        C: g = 2C/dt
//     closed switch: g = 1/R_sw               line end: g = 1/Z_c
//   branch b from node k to node m, v_b = V(k) - V(m), V(ground) = 0,
//   V(source s) = A_s sin(2 pi f_s t_n + phi_s), t_n = n dt:
//     current k->m:  i_b(n) = g v_b(n) + h_b(n-1)      (h = 0 for R)
//     L: h_b(n) = h_b(n-1) + 2 g v_b(n)
//     C: h_b(n) = -h_b(n-1) - 2 g v_b(n)
//   lossless line (k, m), Z_c, travel time d steps (Bergeron):
//     current k->line: v_k(n)/Z_c + I_k(n)
//     I_m(n+d) = -(2/Z_c) v_k(n) - I_k(n),  I_k(n+d) = -(2/Z_c) v_m(n) - I_m(n)
//   nodal equations per step:  G v_n = u_n - A h_{n-1} - L I_n
//
// The time loop starts de-energised: v_0 = 0, h_0 = 0, I(n) = 0 for n <= d,
// and the first solved step is n = 1.  Each conductance matrix is factorised
// by LU with partial pivoting whenever the switch state changes (process 3)
// and every step is a forward/backward substitution (process 4).
//
// The scalar type is a template parameter so the same loop runs in complex
// arithmetic for complex-step derivatives.
#include "emt_oracle.h"

#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace {

using cplx = std::complex<double>;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dense LU

// In-place LU with partial pivoting (Doolittle), row-major n x n.
// Pivots on the magnitude of the real part so that a complex-step run takes
// the same pivot sequence as the real run.
template <class T>
bool lu_factor(int n, std::vector<T>& a, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(re(a[(size_t)k * n + k]));
    for (int i = k + 1; i < n; ++i) {
      double m = std::fabs(re(a[(size_t)i * n + k]));
      if (m > best) { best = m; p = i; }
    }
    if (!(best > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      T f = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= f * a[(size_t)k * n + j];
    }
  }
  return true;
}

// Solve with the factors: apply the row swaps, then L y = Pb, then U x = y.
template <class T>
void lu_solve(int n, const std::vector<T>& lu, const std::vector<int>& piv, T* x) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(x[k], x[piv[k]]);
  for (int i = 0; i < n; ++i) {
    T s = x[i];
    for (int j = 0; j < i; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = x[i];
    for (int j = i + 1; j < n; ++j) s -= lu[(size_t)i * n + j] * x[j];
    x[i] = s / lu[(size_t)i * n + i];
  }
}

// Solve A^T x = b with the factors of P A = L U:  A^T = U^T L^T P,
// so U^T z = b, L^T y = z, x = P^T y.
template <class T>
void lu_solve_transposed(int n, const std::vector<T>& lu, const std::vector<int>& piv, T* x) {
  for (int i = 0; i < n; ++i) {
    T s = x[i];
    for (int j = 0; j < i; ++j) s -= lu[(size_t)j * n + i] * x[j];
    x[i] = s / lu[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = x[i];
    for (int j = i + 1; j < n; ++j) s -= lu[(size_t)j * n + i] * x[j];
    x[i] = s;
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k) std::swap(x[k], x[piv[k]]);
}

// ---------------------------------------------------------------- network

// Inverse of a 3 x 3 row-major matrix by cofactors; false if singular.
bool invert3(const double* a, double* inv) {
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
  inv[0] = c00 / det;
  inv[3] = c01 / det;
  inv[6] = c02 / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  return true;
}

bool valid(const orc_net* net) {
  if (!net || !(net->dt > 0.0) || net->n_nodes < 0) return false;
  auto node_ok = [&](int32_t x) { return x >= -1 - net->n_src && x < net->n_nodes; };
  for (int64_t b = 0; b < net->n_br; ++b) {
    int32_t k = net->br_k[b], m = net->br_m[b];
    if (!node_ok(k) || !node_ok(m) || k == m) return false;
    if (k < 0 && m < 0) return false;
    if (net->br_kind[b] > 2 || !(net->br_val[b] > 0.0) || !std::isfinite(net->br_val[b])) return false;
  }
  for (int64_t l = 0; l < net->n_ln; ++l) {
    if (net->ln_k[l] < 0 || net->ln_m[l] < 0 || net->ln_k[l] >= net->n_nodes || net->ln_m[l] >= net->n_nodes) return false;
    if (net->ln_k[l] == net->ln_m[l] || net->ln_d[l] < 1 || !(net->ln_zc[l] > 0.0)) return false;
  }
  for (int64_t s = 0; s < net->n_sw; ++s) {
    int32_t k = net->sw_k[s], m = net->sw_m[s];
    if (k < -1 || m < -1 || k >= net->n_nodes || m >= net->n_nodes || k == m || (k < 0 && m < 0)) return false;
    if (!(net->sw_r[s] > 0.0)) return false;
  }
  if (net->n_cl < 0) return false;
  for (int64_t l = 0; l < net->n_cl; ++l) {
    for (int p = 0; p < 6; ++p) {
      const int32_t x = p < 3 ? net->cl_k[3 * l + p] : net->cl_m[3 * l + p - 3];
      if (x < 0 || x >= net->n_nodes) return false;
    }
    for (int j = 0; j < 3; ++j)
      if (!(net->cl_z[3 * l + j] > 0.0) || !(net->cl_tau[3 * l + j] >= net->dt) || !std::isfinite(net->cl_tau[3 * l + j]))
        return false;
    double inv[9];
    if (!invert3(net->cl_tv + 9 * l, inv)) return false;
  }
  if (net->n_rs < 0) return false;
  for (int64_t w = 0; w < net->n_rs; ++w) {
    int32_t k = net->rs_k[w], m = net->rs_m[w];
    if (k < -1 || m < -1 || k >= net->n_nodes || m >= net->n_nodes || k == m || (k < 0 && m < 0)) return false;
    if (net->rs_kind[w] > 1 || !(net->rs_ron[w] > 0.0) || !(net->rs_roff[w] > 0.0)) return false;
  }
  if (net->n_fl < 0) return false;
  for (int64_t l = 0; l < net->n_fl; ++l) {
    const int32_t k = net->fl_k[l], m = net->fl_m[l];
    if (k < 0 || m < 0 || k >= net->n_nodes || m >= net->n_nodes || k == m) return false;
    if (!(net->fl_tau[l] >= net->dt) || !std::isfinite(net->fl_tau[l])) return false;
    if (!(net->fl_y0[l] >= 0.0) || !std::isfinite(net->fl_y0[l]) || !std::isfinite(net->fl_a0[l])) return false;
    if (net->fl_ny[l] < 0 || net->fl_ny[l] > 4 || net->fl_na[l] < 0 || net->fl_na[l] > 4) return false;
    double geq = net->fl_y0[l];
    for (int i = 0; i < net->fl_ny[l]; ++i) {
      const double q = net->fl_yq[4 * l + i], c = net->fl_yc[4 * l + i];
      if (!(q < 0.0) || !std::isfinite(q) || !std::isfinite(c)) return false;
      geq += c * (net->dt / 2.0) / (1.0 - q * net->dt / 2.0);
    }
    if (!(geq > 0.0)) return false;
    for (int i = 0; i < net->fl_na[l]; ++i)
      if (!(net->fl_ap[4 * l + i] < 0.0) || !std::isfinite(net->fl_ap[4 * l + i]) ||
          !std::isfinite(net->fl_ar[4 * l + i]))
        return false;
  }
  if (net->n_nl < 0) return false;
  for (int64_t e = 0; e < net->n_nl; ++e) {
    const int32_t k = net->nl_k[e], m = net->nl_m[e];
    if (k < -1 || m < -1 || k >= net->n_nodes || m >= net->n_nodes || k == m || (k < 0 && m < 0)) return false;
    const int np = net->nl_np[e];
    if (np < 1 || np > 8) return false;
    double pv = 0.0, pi = 0.0;
    for (int j = 0; j < np; ++j) {
      const double vj = net->nl_v[8 * e + j], ij = net->nl_i[8 * e + j];
      if (!std::isfinite(vj) || !std::isfinite(ij) || !(vj > pv) || !(ij >= pi)) return false;
      pv = vj;
      pi = ij;
    }
  }
  if (net->n_cb < 0 || net->n_ci < 0) return false;
  for (int64_t b = 0; b < net->n_cb; ++b) {
    const int t = net->cb_type[b];
    if (t > 8 || !std::isfinite(net->cb_p0[b]) || !std::isfinite(net->cb_p1[b])) return false;
    const int n_in = (t <= 1) ? 0 : (t == 3 || t == 4) ? 2 : 1;
    const int32_t in[2] = {net->cb_in0[b], net->cb_in1[b]};
    for (int i = 0; i < n_in; ++i)
      if (in[i] < 0 || in[i] >= net->n_cb) return false;
    if (t == 1 && (net->cb_node[b] < 0 || net->cb_node[b] >= net->n_nodes)) return false;
    if (t == 5 && !(net->cb_p0[b] <= net->cb_p1[b])) return false;
    if (t == 7 && !(net->cb_p1[b] > 0.0)) return false;
  }
  for (int64_t c = 0; c < net->n_ci; ++c)
    if (net->ci_block[c] < 0 || net->ci_block[c] >= net->n_cb || net->ci_node[c] < 0 ||
        net->ci_node[c] >= net->n_nodes)
      return false;
  if (net->n_fg < 0) return false;
  std::vector<char> grouped(net->n_fl > 0 ? net->n_fl : 0, 0);
  for (int64_t g = 0; g < net->n_fg; ++g) {
    for (int j = 0; j < 3; ++j) {
      const int32_t l = net->fg_line[3 * g + j];
      if (l < 0 || l >= net->n_fl || grouped[l]) return false;
      grouped[l] = 1;
    }
    double inv[9];
    if (!invert3(net->fg_tv + 9 * g, inv)) return false;
  }
  return true;
}

// Connected components of unknown nodes over branches and switches
// (ground and source nodes do not join anything; lines are cuts).
int find(std::vector<int>& p, int x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

void components(const orc_net* net, std::vector<int>& sub, int& n_sub) {
  int n = (int)net->n_nodes;
  std::vector<int> p(n);
  for (int i = 0; i < n; ++i) p[i] = i;
  auto join = [&](int a, int b) {
    if (a < 0 || b < 0) return;
    a = find(p, a); b = find(p, b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  };
  for (int64_t b = 0; b < net->n_br; ++b) join(net->br_k[b], net->br_m[b]);
  for (int64_t s = 0; s < net->n_sw; ++s) join(net->sw_k[s], net->sw_m[s]);
  for (int64_t w = 0; w < net->n_rs; ++w) join(net->rs_k[w], net->rs_m[w]);
  for (int64_t e = 0; e < net->n_nl; ++e) join(net->nl_k[e], net->nl_m[e]);
  for (int64_t l = 0; l < net->n_cl; ++l)
    for (int p = 1; p < 3; ++p) {
      join(net->cl_k[3 * l], net->cl_k[3 * l + p]);
      join(net->cl_m[3 * l], net->cl_m[3 * l + p]);
    }
  for (int64_t g = 0; g < net->n_fg; ++g)   // a group end's three phase nodes are coupled
    for (int p = 1; p < 3; ++p) {
      join(net->fl_k[net->fg_line[3 * g]], net->fl_k[net->fg_line[3 * g + p]]);
      join(net->fl_m[net->fg_line[3 * g]], net->fl_m[net->fg_line[3 * g + p]]);
    }
  sub.assign(n, -1);
  n_sub = 0;
  std::vector<int> label(n, -1);
  for (int i = 0; i < n; ++i) {
    int r = find(p, i);
    if (label[r] < 0) label[r] = n_sub++;
    sub[i] = label[r];
  }
}

template <class T>
T conductance(uint8_t kind, const T& value, double dt) {
  if (kind == 0) return T(1.0) / value;
  if (kind == 1) return T(dt) / (T(2.0) * value);
  return T(2.0) * value / T(dt);
}

bool switch_closed(const orc_net* net, int64_t s, int64_t n) {
  return net->sw_on[s] >= 0 && n >= net->sw_on[s] && (net->sw_off[s] < 0 || n < net->sw_off[s]);
}

// One simulation.  Parameters (branch values, source amplitudes) are given
// in the scalar type T so that complex-step runs can perturb one of them.
template <class T>
struct Sim {
  const orc_net* net;
  int n_nodes;
  std::vector<T> g;          // companion conductance per branch
  std::vector<T> amp;        // source amplitudes
  std::vector<int> sub;      // subsystem of each unknown node
  int n_sub = 0;
  std::vector<std::vector<int>> nodes;   // nodes of each subsystem
  std::vector<int> local;                // local index of each node
  std::vector<std::vector<T>> lu;        // factors per subsystem (current switch state)
  std::vector<std::vector<int>> piv;
  std::vector<std::vector<char>> state;  // switch state the factors belong to
  std::vector<T> h;                      // history current per branch
  // line history rings: I value consumed at end k (slot 0) / end m (slot 1)
  // of line l at step n lives at ring[l][end][n mod (d+1)]
  std::vector<std::vector<T>> ring_k, ring_m;
  std::vector<T> vsrc;   // source voltages at the current step
  std::vector<T> v;      // node voltages at the current step
  std::vector<char> rs_on;     // runtime-switch state in force at the current step
  std::vector<double> rs_i;    // breaker current of the previous step
  // coupled lines: per line T_v^-1, T_i, Y_p (3 x 3), per mode d, f, 2/Z;
  // c values each end sent, by step modulo d + 2: cl_c[line][end][mode]
  struct CLine {
    double tinv[9], ti[9], yp[9], y2[3], f[3];
    int64_t d[3];
    std::vector<T> c[2][3];
    T im[2][3];   // modal history currents of the current step per end
  };
  std::vector<CLine> cl;
  // frequency-dependent lines: per line the discretised terms, per end the
  // states, the values w each end sent (by step modulo d + 3) and W of the
  // previous step
  struct FLine {
    int64_t d;
    double phi, geq, y0, a0;
    int ny, na;
    double lam_y[4], mu_y[4], lam_a[4], mu_a[4];
    T s[2][4], z[2][4], vprev[2], wprev[2], b[2];
    std::vector<T> w[2];
  };
  std::vector<FLine> fl;
  // frequency-dependent line groups: T_v^-1 and T_i of each; per line its
  // group (or -1) and mode
  struct FGroup {
    double tinv[9], ti[9];
  };
  std::vector<FGroup> fg;
  std::vector<int> fl_grp, fl_mode;
  // nonlinear resistors: the one of each subsystem (or -1) and its column
  // z = G^-1 (e_k - e_m) over the subsystem's nodes, for the current factors
  std::vector<int> nl_of_sub;                  // the subsystem's nonlinear resistor when it has exactly one, else -1
  std::vector<std::vector<T>> nl_z;
  std::vector<std::vector<int64_t>> nl_list;   // all nonlinear resistors of each subsystem
  std::vector<std::vector<T>> gmat;            // unfactorised G of subsystems with several of them
  std::vector<int> nl_seg;                     // per nonlinear resistor: segment of the last step, sign * (j + 1)
  // control blocks: output of the latest evaluation, and the two states
  // (integral or previous output; previous input)
  std::vector<T> cy, cs0, cs1;
  // subsystems whose processes 3 and 4 run (empty: all); see orc_advance
  std::vector<char> active;

  bool init(const T* br_value, const T* src_amp, bool monolithic) {
    n_nodes = (int)net->n_nodes;
    g.resize(net->n_br);
    for (int64_t b = 0; b < net->n_br; ++b) g[b] = conductance<T>(net->br_kind[b], br_value[b], net->dt);
    amp.assign(src_amp, src_amp + net->n_src);
    if (monolithic) {
      sub.assign(n_nodes, 0);
      n_sub = n_nodes > 0 ? 1 : 0;
    } else {
      components(net, sub, n_sub);
    }
    nodes.assign(n_sub, {});
    local.assign(n_nodes, -1);
    for (int i = 0; i < n_nodes; ++i) {
      local[i] = (int)nodes[sub[i]].size();
      nodes[sub[i]].push_back(i);
    }
    lu.assign(n_sub, {});
    piv.assign(n_sub, {});
    state.assign(n_sub, {});
    h.assign(net->n_br, T(0.0));
    ring_k.assign(net->n_ln, {});
    ring_m.assign(net->n_ln, {});
    for (int64_t l = 0; l < net->n_ln; ++l) {
      ring_k[l].assign(net->ln_d[l] + 1, T(0.0));
      ring_m[l].assign(net->ln_d[l] + 1, T(0.0));
    }
    vsrc.assign(net->n_src, T(0.0));
    v.assign(n_nodes, T(0.0));
    rs_on.assign(net->n_rs, 0);
    for (int64_t w = 0; w < net->n_rs; ++w) rs_on[w] = net->rs_on0[w] ? 1 : 0;
    rs_i.assign(net->n_rs, 0.0);
    nl_of_sub.assign(n_sub, -1);
    nl_z.assign(n_sub, {});
    nl_list.assign(n_sub, {});
    gmat.assign(n_sub, {});
    nl_seg.assign(net->n_nl, 1);
    for (int64_t e = 0; e < net->n_nl; ++e) {
      const int a = net->nl_k[e] >= 0 ? net->nl_k[e] : net->nl_m[e];
      nl_list[sub[a]].push_back(e);
    }
    for (int s = 0; s < n_sub; ++s)
      if (nl_list[s].size() == 1) nl_of_sub[s] = (int)nl_list[s][0];
    fl.assign(net->n_fl, FLine{});
    for (int64_t l = 0; l < net->n_fl; ++l) {
      FLine& L = fl[l];
      const double dt = net->dt, steps = net->fl_tau[l] / dt;
      L.d = (int64_t)std::floor(steps);
      L.phi = steps - (double)L.d;
      L.y0 = net->fl_y0[l];
      L.a0 = net->fl_a0[l];
      L.ny = net->fl_ny[l];
      L.na = net->fl_na[l];
      L.geq = L.y0;
      for (int i = 0; i < L.ny; ++i) {
        const double q = net->fl_yq[4 * l + i], den = 1.0 - q * dt / 2.0;
        L.lam_y[i] = (1.0 + q * dt / 2.0) / den;
        L.mu_y[i] = net->fl_yc[4 * l + i] * (dt / 2.0) / den;
        L.geq += L.mu_y[i];
      }
      for (int i = 0; i < L.na; ++i) {
        const double p = net->fl_ap[4 * l + i], den = 1.0 - p * dt / 2.0;
        L.lam_a[i] = (1.0 + p * dt / 2.0) / den;
        L.mu_a[i] = net->fl_ar[4 * l + i] * (dt / 2.0) / den;
      }
      for (int e = 0; e < 2; ++e) {
        for (int i = 0; i < 4; ++i) L.s[e][i] = L.z[e][i] = T(0.0);
        L.vprev[e] = L.wprev[e] = L.b[e] = T(0.0);
        L.w[e].assign(L.d + 3, T(0.0));
      }
    }
    fg.assign(net->n_fg, FGroup{});
    fl_grp.assign(net->n_fl, -1);
    fl_mode.assign(net->n_fl, 0);
    for (int64_t gi = 0; gi < net->n_fg; ++gi) {
      FGroup& G = fg[gi];
      invert3(net->fg_tv + 9 * gi, G.tinv);
      for (int p = 0; p < 3; ++p)
        for (int j = 0; j < 3; ++j) G.ti[3 * p + j] = G.tinv[3 * j + p];   // T_i = (T_v^-1)^T
      for (int j = 0; j < 3; ++j) {
        fl_grp[net->fg_line[3 * gi + j]] = (int)gi;
        fl_mode[net->fg_line[3 * gi + j]] = j;
      }
    }
    cy.assign(net->n_cb, T(0.0));
    cs0.assign(net->n_cb, T(0.0));
    cs1.assign(net->n_cb, T(0.0));
    cl.assign(net->n_cl, CLine{});
    for (int64_t l = 0; l < net->n_cl; ++l) {
      CLine& L = cl[l];
      invert3(net->cl_tv + 9 * l, L.tinv);
      for (int p = 0; p < 3; ++p)
        for (int j = 0; j < 3; ++j) L.ti[3 * p + j] = L.tinv[3 * j + p];   // T_i = (T_v^-1)^T
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
          double acc = 0.0;
          for (int j = 0; j < 3; ++j) acc += L.ti[3 * p + j] * (1.0 / net->cl_z[3 * l + j]) * L.tinv[3 * j + q];
          L.yp[3 * p + q] = acc;
        }
      for (int j = 0; j < 3; ++j) {
        const double steps = net->cl_tau[3 * l + j] / net->dt;
        L.d[j] = (int64_t)std::floor(steps);
        L.f[j] = steps - (double)L.d[j];
        L.y2[j] = 2.0 / net->cl_z[3 * l + j];
        for (int e = 0; e < 2; ++e) L.c[e][j].assign(L.d[j] + 2, T(0.0));
      }
    }
    return true;
  }

  // c value end e of coupled line L sent at step m (0 before the start)
  T cl_sent(const CLine& L, int e, int j, int64_t m) const {
    if (m < 1) return T(0.0);
    return L.c[e][j][m % (L.d[j] + 2)];
  }

  // Runtime switches: the states in force at step n+1 from step n's solution.
  void decide_runtime_switches(int64_t n) {
    for (int64_t w = 0; w < net->n_rs; ++w) {
      const double vb = re(node_voltage(net->rs_k[w])) - re(node_voltage(net->rs_m[w]));
      if (net->rs_kind[w] == 0) {
        rs_on[w] = vb > 0.0 ? 1 : 0;
      } else if (rs_on[w]) {
        const double i = vb / net->rs_ron[w];
        if (n >= net->rs_trip[w] && rs_i[w] * i <= 0.0) rs_on[w] = 0;
        rs_i[w] = i;
      }
    }
  }

  // w value end e of frequency-dependent line L sent at step m (0 before the start)
  T fl_sent(const FLine& L, int e, int64_t m) const {
    if (m < 1) return T(0.0);
    return L.w[e][m % (L.d + 3)];
  }

  // Control blocks at step n, in index order over one array: an input of
  // lower index has already been overwritten with its step-n output, one of
  // equal or higher index still holds step n-1's.
  void evaluate_controls() {
    const double dt = net->dt;
    for (int64_t b = 0; b < net->n_cb; ++b) {
      const double p0 = net->cb_p0[b], p1 = net->cb_p1[b];
      const T u0 = net->cb_in0[b] >= 0 ? cy[net->cb_in0[b]] : T(0.0);
      const T u1 = net->cb_in1[b] >= 0 ? cy[net->cb_in1[b]] : T(0.0);
      T y;
      switch (net->cb_type[b]) {
        case 0: y = T(p0); break;
        case 1: y = v[net->cb_node[b]]; break;
        case 2: y = T(p0) * u0; break;
        case 3: y = T(p0) * u0 + T(p1) * u1; break;
        case 4: y = T(p0) * u0 * u1; break;
        case 5: y = re(u0) < p0 ? T(p0) : (re(u0) > p1 ? T(p1) : u0); break;
        case 6:
          y = cs0[b] + T(p0 * (dt / 2.0)) * (u0 + cs1[b]);
          cs0[b] = y;
          cs1[b] = u0;
          break;
        case 7: {
          const double a = (2.0 * p1 - dt) / (2.0 * p1 + dt), bb = p0 * dt / (2.0 * p1 + dt);
          y = T(a) * cs0[b] + T(bb) * (u0 + cs1[b]);
          cs0[b] = y;
          cs1[b] = u0;
          break;
        }
        default: {   // 8: PI
          const T integral = cs0[b] + T(dt / 2.0) * (u0 + cs1[b]);
          y = T(p0) * u0 + T(p1) * integral;
          cs0[b] = integral;
          cs1[b] = u0;
          break;
        }
      }
      cy[b] = y;
    }
  }

  // Process 3: assemble the subsystem's conductance matrix for the switch
  // state of step n and factorise it, if that state differs from the one
  // the current factors belong to.
  bool refactor_if_needed(int s, int64_t n) {
    std::vector<char> st(net->n_sw + net->n_rs, 0);
    for (int64_t w = 0; w < net->n_sw; ++w) {
      int a = net->sw_k[w] >= 0 ? net->sw_k[w] : net->sw_m[w];
      if (sub[a] == s) st[w] = switch_closed(net, w, n) ? 1 : 0;
    }
    for (int64_t w = 0; w < net->n_rs; ++w) {
      int a = net->rs_k[w] >= 0 ? net->rs_k[w] : net->rs_m[w];
      if (sub[a] == s) st[net->n_sw + w] = rs_on[w];
    }
    if (!lu[s].empty() && st == state[s]) return true;
    state[s] = st;
    int ns = (int)nodes[s].size();
    std::vector<T> G((size_t)ns * ns, T(0.0));
    auto stamp = [&](int32_t k, int32_t m, const T& gg) {
      int a = (k >= 0) ? local[k] : -1;
      int b = (m >= 0) ? local[m] : -1;
      if (a >= 0) G[(size_t)a * ns + a] += gg;
      if (b >= 0) G[(size_t)b * ns + b] += gg;
      if (a >= 0 && b >= 0) {
        G[(size_t)a * ns + b] -= gg;
        G[(size_t)b * ns + a] -= gg;
      }
    };
    for (int64_t b = 0; b < net->n_br; ++b) {
      int32_t k = net->br_k[b], m = net->br_m[b];
      int a = k >= 0 ? k : m;
      if (sub[a] != s) continue;
      stamp(k, m, g[b]);   // a source end acts like ground in G
    }
    for (int64_t l = 0; l < net->n_ln; ++l) {
      T y = T(1.0) / T(net->ln_zc[l]);
      if (sub[net->ln_k[l]] == s) G[(size_t)local[net->ln_k[l]] * ns + local[net->ln_k[l]]] += y;
      if (sub[net->ln_m[l]] == s) G[(size_t)local[net->ln_m[l]] * ns + local[net->ln_m[l]]] += y;
    }
    for (int64_t l = 0; l < net->n_fl; ++l) {
      if (fl_grp[l] >= 0) continue;   // (groups below)
      for (int32_t x : {net->fl_k[l], net->fl_m[l]})
        if (sub[x] == s) G[(size_t)local[x] * ns + local[x]] += T(fl[l].geq);
    }
    for (int64_t gi = 0; gi < net->n_fg; ++gi)   // each end: T_i diag(G_eq) T_v^-1 over its phase nodes
      for (int e = 0; e < 2; ++e) {
        const FGroup& F = fg[gi];
        int32_t nd[3];
        for (int p = 0; p < 3; ++p) nd[p] = e == 0 ? net->fl_k[net->fg_line[3 * gi + p]] : net->fl_m[net->fg_line[3 * gi + p]];
        if (sub[nd[0]] != s) continue;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += F.ti[3 * p + j] * fl[net->fg_line[3 * gi + j]].geq * F.tinv[3 * j + q];
            G[(size_t)local[nd[p]] * ns + local[nd[q]]] += T(acc);
          }
      }
    for (int64_t w = 0; w < net->n_sw; ++w)
      if (st[w]) stamp(net->sw_k[w], net->sw_m[w], T(1.0) / T(net->sw_r[w]));
    for (int64_t w = 0; w < net->n_rs; ++w) {
      int a = net->rs_k[w] >= 0 ? net->rs_k[w] : net->rs_m[w];
      if (sub[a] == s) stamp(net->rs_k[w], net->rs_m[w], T(1.0) / T(rs_on[w] ? net->rs_ron[w] : net->rs_roff[w]));
    }
    for (int64_t l = 0; l < net->n_cl; ++l)
      for (int e = 0; e < 2; ++e) {
        const int32_t* nd = (e == 0 ? net->cl_k : net->cl_m) + 3 * l;
        if (sub[nd[0]] != s) continue;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) G[(size_t)local[nd[p]] * ns + local[nd[q]]] += T(cl[l].yp[3 * p + q]);
      }
    lu[s] = G;
    if (nl_list[s].size() > 1) gmat[s] = G;
    if (!lu_factor(ns, lu[s], piv[s])) return false;
    if (nl_of_sub[s] >= 0) {   // the nonlinear resistor's column G^-1 (e_k - e_m)
      const int64_t e = nl_of_sub[s];
      std::vector<T> z(ns, T(0.0));
      if (net->nl_k[e] >= 0) z[local[net->nl_k[e]]] += T(1.0);
      if (net->nl_m[e] >= 0) z[local[net->nl_m[e]]] -= T(1.0);
      lu_solve(ns, lu[s], piv[s], z.data());
      nl_z[s] = z;
    }
    return true;
  }

  // The current of nonlinear resistor e from its Thevenin source v_th behind
  // r_th: the unique i with i = f(v_th - r_th i), f odd and piecewise linear
  // (the segment whose image under u -> u + r_th f(u) holds |v_th|).
  T nl_current(int64_t e, const T& v_th, const T& r_th) const {
    const double* pv = net->nl_v + 8 * e;
    const double* pi = net->nl_i + 8 * e;
    const int np = net->nl_np[e];
    const double sgn = re(v_th) < 0.0 ? -1.0 : 1.0;
    const T x = T(sgn) * v_th;   // |v_th|
    double v0 = 0.0, i0 = 0.0, slope = 0.0;
    int j = 0;
    for (; j < np; ++j) {
      slope = (pi[j] - i0) / (pv[j] - v0);
      if (re(x) < pv[j] + re(r_th) * pi[j]) break;   // the image of breakpoint j
      v0 = pv[j];
      i0 = pi[j];
    }
    // on the segment from (v0, i0) with this slope (past the last point the
    // last segment's slope): u + r_th (i0 + slope (u - v0)) = |v_th|
    const T u = (x - r_th * T(i0 - slope * v0)) / (T(1.0) + r_th * T(slope));
    return T(sgn) * (T(i0) + T(slope) * (u - T(v0)));
  }

  // Segment of nonlinear resistor e that holds the voltage u: sign(u) * (j + 1),
  // j = the number of breakpoints at or below |u| (j = np: past the last one).
  int nl_segment_of(int64_t e, double u) const {
    const double* pv = net->nl_v + 8 * e;
    const int np = net->nl_np[e];
    const double x = std::fabs(u);
    int j = 0;
    while (j < np && x >= pv[j]) ++j;
    return u < 0.0 ? -(j + 1) : j + 1;
  }

  // The line i = c0 + slope u of f on segment code sg (see nl_segment_of):
  // from (v0, i0), the segment's start, with the segment's slope (past the
  // last breakpoint the last slope); odd: i = sign (i0 + slope (sign u - v0)).
  void nl_line(int64_t e, int sg, double& slope, double& c0) const {
    const double* pv = net->nl_v + 8 * e;
    const double* pi = net->nl_i + 8 * e;
    const int np = net->nl_np[e];
    const double sgn = sg < 0 ? -1.0 : 1.0;
    const int j = (sg < 0 ? -sg : sg) - 1;
    double v0 = 0.0, i0 = 0.0, sl = 0.0;
    for (int q = 0; q < np && q <= j; ++q) {   // walk the segments up to j, as nl_current does
      sl = (pi[q] - i0) / (pv[q] - v0);
      if (q == j) break;
      v0 = pv[q];
      i0 = pi[q];
    }
    slope = sl;
    c0 = sgn * (i0 - sl * v0);
  }

  T node_voltage(int32_t x) const {
    if (x >= 0) return v[x];
    if (x == -1) return T(0.0);
    return vsrc[-2 - x];
  }

  // One time step n >= 1.  Returns false if a matrix is singular.
  bool step(int64_t n) {
    const double t = (double)n * net->dt;
    for (int64_t s = 0; s < net->n_src; ++s)
      vsrc[s] = amp[s] * std::sin(2.0 * kPi * net->src_freq[s] * t + net->src_phase[s]);
    // process 2: nodal injections u_n - A h_{n-1} - L I_n
    std::vector<T> rhs(n_nodes, T(0.0));
    for (int64_t b = 0; b < net->n_br; ++b) {
      int32_t k = net->br_k[b], m = net->br_m[b];
      if (k >= 0 && m <= -2) rhs[k] += g[b] * vsrc[-2 - m];
      if (m >= 0 && k <= -2) rhs[m] += g[b] * vsrc[-2 - k];
      if (net->br_kind[b] != 0) {
        if (k >= 0) rhs[k] -= h[b];
        if (m >= 0) rhs[m] += h[b];
      }
    }
    for (int64_t c = 0; c < net->n_ci; ++c) rhs[net->ci_node[c]] += cy[net->ci_block[c]];   // y(n-1)
    // frequency-dependent lines: the far end's interpolated w, A's terms,
    // and the history current each end draws
    std::vector<T> fhist(2 * (size_t)net->n_fl, T(0.0));   // per line and end: the history current drawn
    for (int64_t l = 0; l < net->n_fl; ++l) {
      FLine& L = fl[l];
      for (int e = 0; e < 2; ++e) {
        const T W = T(1.0 - L.phi) * fl_sent(L, 1 - e, n - L.d) + T(L.phi) * fl_sent(L, 1 - e, n - L.d - 1);
        T b = T(L.a0) * W;
        for (int i = 0; i < L.na; ++i) {
          L.z[e][i] = T(L.lam_a[i]) * L.z[e][i] + T(L.mu_a[i]) * (W + L.wprev[e]);
          b += L.z[e][i];
        }
        L.wprev[e] = W;
        L.b[e] = b;
        T hist = -b;
        for (int i = 0; i < L.ny; ++i) hist += T(L.lam_y[i]) * L.s[e][i] + T(L.mu_y[i]) * L.vprev[e];
        fhist[2 * l + e] = hist;
        if (fl_grp[l] < 0) rhs[e == 0 ? net->fl_k[l] : net->fl_m[l]] -= hist;
      }
    }
    // line groups: the modal history currents enter the phase nodes as T_i hist_mode
    for (int64_t gi = 0; gi < net->n_fg; ++gi)
      for (int e = 0; e < 2; ++e)
        for (int p = 0; p < 3; ++p) {
          const int32_t lp = net->fg_line[3 * gi + p];
          T ip = T(0.0);
          for (int j = 0; j < 3; ++j) ip += T(fg[gi].ti[3 * p + j]) * fhist[2 * net->fg_line[3 * gi + j] + e];
          rhs[e == 0 ? net->fl_k[lp] : net->fl_m[lp]] -= ip;
        }
    for (int64_t l = 0; l < net->n_ln; ++l) {
      int64_t d1 = net->ln_d[l] + 1;
      rhs[net->ln_k[l]] -= ring_k[l][n % d1];
      rhs[net->ln_m[l]] -= ring_m[l][n % d1];
    }
    // coupled lines: modal histories from the far end's sent values, then
    // phase-domain history currents T_i I_mode leaving each end's nodes
    for (int64_t l = 0; l < net->n_cl; ++l) {
      CLine& L = cl[l];
      for (int e = 0; e < 2; ++e) {
        for (int j = 0; j < 3; ++j)
          L.im[e][j] = T(1.0 - L.f[j]) * cl_sent(L, 1 - e, j, n - L.d[j]) +
                       T(L.f[j]) * cl_sent(L, 1 - e, j, n - L.d[j] - 1);
        const int32_t* nd = (e == 0 ? net->cl_k : net->cl_m) + 3 * l;
        for (int p = 0; p < 3; ++p) {
          T ip = T(0.0);
          for (int j = 0; j < 3; ++j) ip += T(L.ti[3 * p + j]) * L.im[e][j];
          rhs[nd[p]] -= ip;
        }
      }
    }
    // processes 3 and 4 per subsystem
    for (int s = 0; s < n_sub; ++s) {
      if (!active.empty() && !active[s]) continue;
      if (!refactor_if_needed(s, n)) return false;
      int ns = (int)nodes[s].size();
      std::vector<T> x(ns);
      for (int i = 0; i < ns; ++i) x[i] = rhs[nodes[s][i]];
      lu_solve(ns, lu[s], piv[s], x.data());
      if (nl_of_sub[s] >= 0) {   // compensation: the nonlinear resistor against the linear solution
        const int64_t e = nl_of_sub[s];
        const int32_t k = net->nl_k[e], m = net->nl_m[e];
        const std::vector<T>& z = nl_z[s];
        const T vth = (k >= 0 ? x[local[k]] : T(0.0)) - (m >= 0 ? x[local[m]] : T(0.0));
        const T rth = (k >= 0 ? z[local[k]] : T(0.0)) - (m >= 0 ? z[local[m]] : T(0.0));
        const T inl = nl_current(e, vth, rth);
        for (int i = 0; i < ns; ++i) x[i] -= z[i] * inl;
      } else if (nl_list[s].size() > 1) {
        // several nonlinear resistors: the piecewise-linear Newton iteration on
        // the subsystem's nodal equations, from the previous step's segments:
        // every element stamped as its segment's line i = c0 + slope u, the
        // system solved, every element moved to the segment its voltage lies
        // on, until no element moves (f monotone: the solution is unique)
        bool settled = false;
        for (int it = 0; it < 64 && !settled; ++it) {
          std::vector<T> Gs = gmat[s];
          std::vector<int> ps(ns);
          for (int i = 0; i < ns; ++i) x[i] = rhs[nodes[s][i]];
          for (int64_t e : nl_list[s]) {
            double slope, c0;
            nl_line(e, nl_seg[e], slope, c0);
            const int a = net->nl_k[e] >= 0 ? local[net->nl_k[e]] : -1;
            const int b = net->nl_m[e] >= 0 ? local[net->nl_m[e]] : -1;
            if (a >= 0) {
              Gs[(size_t)a * ns + a] += T(slope);
              x[a] -= T(c0);
            }
            if (b >= 0) {
              Gs[(size_t)b * ns + b] += T(slope);
              x[b] += T(c0);
            }
            if (a >= 0 && b >= 0) {
              Gs[(size_t)a * ns + b] -= T(slope);
              Gs[(size_t)b * ns + a] -= T(slope);
            }
          }
          if (!lu_factor(ns, Gs, ps)) return false;
          lu_solve(ns, Gs, ps, x.data());
          settled = true;
          for (int64_t e : nl_list[s]) {
            const int32_t k = net->nl_k[e], m = net->nl_m[e];
            const double u = re((k >= 0 ? x[local[k]] : T(0.0)) - (m >= 0 ? x[local[m]] : T(0.0)));
            const int sg = nl_segment_of(e, u);
            if (sg != nl_seg[e]) {
              nl_seg[e] = sg;
              settled = false;
            }
          }
        }
        if (!settled) return false;
      }
      for (int i = 0; i < ns; ++i) v[nodes[s][i]] = x[i];
    }
    // process 1: history currents of L and C branches
    for (int64_t b = 0; b < net->n_br; ++b) {
      if (net->br_kind[b] == 0) continue;
      T vb = node_voltage(net->br_k[b]) - node_voltage(net->br_m[b]);
      if (net->br_kind[b] == 1) h[b] = h[b] + T(2.0) * g[b] * vb;
      else h[b] = -h[b] - T(2.0) * g[b] * vb;
    }
    // process 1 for lines: values consumed d steps later at the far ends
    for (int64_t l = 0; l < net->n_ln; ++l) {
      int64_t d = net->ln_d[l], d1 = d + 1;
      T y2 = T(2.0) / T(net->ln_zc[l]);
      T ik = ring_k[l][n % d1], im = ring_m[l][n % d1];
      ring_m[l][(n + d) % d1] = -y2 * v[net->ln_k[l]] - ik;
      ring_k[l][(n + d) % d1] = -y2 * v[net->ln_m[l]] - im;
    }
    // coupled lines: each end sends c_j(n) = -(2/Z_j) v_mode_j(n) - I_mode_j(n)
    for (int64_t l = 0; l < net->n_cl; ++l) {
      CLine& L = cl[l];
      for (int e = 0; e < 2; ++e) {
        const int32_t* nd = (e == 0 ? net->cl_k : net->cl_m) + 3 * l;
        for (int j = 0; j < 3; ++j) {
          T vm = T(0.0);
          for (int p = 0; p < 3; ++p) vm += T(L.tinv[3 * j + p]) * v[nd[p]];
          L.c[e][j][n % (L.d[j] + 2)] = -T(L.y2[j]) * vm - L.im[e][j];
        }
      }
    }
    for (int64_t l = 0; l < net->n_fl; ++l) {
      FLine& L = fl[l];
      for (int e = 0; e < 2; ++e) {
        T ve = v[e == 0 ? net->fl_k[l] : net->fl_m[l]];
        if (fl_grp[l] >= 0) {   // a mode: the modal voltage (T_v^-1 v_phase)_j
          const int gi = fl_grp[l], j = fl_mode[l];
          ve = T(0.0);
          for (int p = 0; p < 3; ++p) {
            const int32_t lp = net->fg_line[3 * gi + p];
            ve += T(fg[gi].tinv[3 * j + p]) * v[e == 0 ? net->fl_k[lp] : net->fl_m[lp]];
          }
        }
        T yc = T(L.y0) * ve;
        for (int i = 0; i < L.ny; ++i) {
          L.s[e][i] = T(L.lam_y[i]) * L.s[e][i] + T(L.mu_y[i]) * (ve + L.vprev[e]);
          yc += L.s[e][i];
        }
        L.w[e][n % (L.d + 3)] = T(2.0) * yc - L.b[e];
        L.vprev[e] = ve;
      }
    }
    evaluate_controls();
    decide_runtime_switches(n);
    return true;
  }
};

template <class T>
int run_loss(const orc_net* net, bool monolithic, int64_t n_steps, const T* br_value, const T* src_amp,
             const int32_t* rec, int64_t n_rec, double* v_out, const double* v_target, T* loss) {
  Sim<T> sim;
  sim.net = net;
  if (!sim.init(br_value, src_amp, monolithic)) return -1;
  T J = T(0.0);
  for (int64_t n = 1; n <= n_steps; ++n) {
    if (!sim.step(n)) return -2;
    if (v_out) {
      double* row = v_out + (size_t)(n - 1) * (rec ? n_rec : net->n_nodes);
      if (rec)
        for (int64_t c = 0; c < n_rec; ++c) row[c] = re(sim.v[rec[c]]);
      else
        for (int64_t k = 0; k < net->n_nodes; ++k) row[k] = re(sim.v[k]);
    }
    if (v_target && loss) {
      const double* tg = v_target + (size_t)(n - 1) * net->n_nodes;
      for (int64_t k = 0; k < net->n_nodes; ++k) {
        T e = sim.v[k] - T(tg[k]);
        J += e * e;
      }
    }
  }
  if (loss) *loss = J;
  return 0;
}

}  // namespace

extern "C" int orc_run(const orc_net* net, int monolithic, int64_t n_steps, const int32_t* rec, int64_t n_rec,
                       double* v_out, const double* v_target, double* loss) {
  if (!valid(net) || n_steps < 0) return -1;
  if (rec)
    for (int64_t c = 0; c < n_rec; ++c)
      if (rec[c] < 0 || rec[c] >= net->n_nodes) return -1;
  return run_loss<double>(net, monolithic != 0, n_steps, net->br_val, net->src_amp, rec, n_rec, v_out,
                          v_target, loss);
}

extern "C" int orc_loss_cs(const orc_net* net, int64_t n_steps, const double* v_target, int64_t param, double h,
                           double* loss, double* dloss) {
  if (!valid(net) || !v_target || param < 0 || param >= net->n_br + net->n_src) return -1;
  std::vector<cplx> bv(net->br_val, net->br_val + net->n_br);
  std::vector<cplx> am(net->src_amp, net->src_amp + net->n_src);
  if (param < net->n_br) bv[param] += cplx(0.0, h);
  else am[param - net->n_br] += cplx(0.0, h);
  cplx J;
  int rc = run_loss<cplx>(net, false, n_steps, bv.data(), am.data(), nullptr, 0, nullptr, v_target, &J);
  if (rc) return rc;
  *loss = J.real();
  *dloss = J.imag() / h;
  return 0;
}

// Reverse-mode (discrete adjoint) of the loop above for
//   J = sum_{n=1..N} sum_k (v_n[k] - v*_n[k])^2.
// With w_n = G_n^{-T} vbar_n, the reverse recursion for n = N..1 is
//   vbar_n      = 2 (v_n - v*_n) + A E hbar_n + (line terms from I(n+d))
//   hbar_{n-1}  = D hbar_n - A^T w_n
//   Ibar_e(n)   = -w_n[k_e] - Ibar_f(n+d)        (f = far end of e)
// where h_n = D h_{n-1} + E v_b(n), D = +1 (L) / -1 (C), E = 2g (L) / -2g (C).
// Parameter terms per step:
//   dJ/dg_b += -(a_b^T w_n) v_b(n) + hbar_n[b] (dE_b/dg_b) v_b(n)
//   dJ/dv_s += g_b w_n[unknown end] + (-/+) E_b hbar_n[b]   (source branches)
//   dJ/dA_s += sin(2 pi f t_n + phi) dJ/dv_s
// and finally dg/dR = -1/R^2, dg/dL = -dt/(2L^2), dg/dC = 2/dt.
extern "C" int orc_adjoint(const orc_net* net, int64_t n_steps, const double* v_target, double* grad,
                           double* loss) {
  if (!valid(net) || !v_target || !grad || n_steps < 0 || net->n_cb > 0 || net->n_fl > 0 || net->n_nl > 0) return -1;
  const int64_t nn = net->n_nodes, nb = net->n_br, ns = net->n_src, nl = net->n_ln, nr = net->n_rs;
  Sim<double> sim;
  sim.net = net;
  if (!sim.init(net->br_val, net->src_amp, false)) return -1;
  std::vector<double> tape((size_t)n_steps * nn);
  // runtime-switch states in force at each step: the reverse sweep uses
  // the matrices the forward run used (decisions held fixed)
  std::vector<char> rs_tape((size_t)n_steps * nr);
  double J = 0.0;
  for (int64_t n = 1; n <= n_steps; ++n) {
    for (int64_t w = 0; w < nr; ++w) rs_tape[(size_t)(n - 1) * nr + w] = sim.rs_on[w];
    if (!sim.step(n)) return -2;
    double* row = tape.data() + (size_t)(n - 1) * nn;
    const double* tg = v_target + (size_t)(n - 1) * nn;
    for (int64_t k = 0; k < nn; ++k) {
      row[k] = sim.v[k];
      double e = sim.v[k] - tg[k];
      J += e * e;
    }
  }
  if (loss) *loss = J;

  std::vector<double> dg(nb, 0.0), dA(ns, 0.0), hbar(nb, 0.0), vbar(nn), w(nn), vs(ns);
  std::vector<std::vector<double>> ibar_k(nl), ibar_m(nl);   // rings, slot n mod (d+1)
  for (int64_t l = 0; l < nl; ++l) {
    ibar_k[l].assign(net->ln_d[l] + 1, 0.0);
    ibar_m[l].assign(net->ln_d[l] + 1, 0.0);
  }
  // coupled lines: adjoints Ibar of the modal histories per end and mode,
  // by step modulo d + 2 (zero beyond the last step); the adjoint of the
  // value c_e,j(n) an end sent is X = (1 - f) Ibar_far(n + d) + f Ibar_far(n + d + 1)
  const int64_t ncl = net->n_cl;
  std::vector<std::vector<double>> cl_ibar((size_t)ncl * 6);
  std::vector<double> cl_x((size_t)ncl * 6, 0.0);
  for (int64_t l = 0; l < ncl; ++l)
    for (int e = 0; e < 2; ++e)
      for (int j = 0; j < 3; ++j) cl_ibar[6 * l + 3 * e + j].assign(sim.cl[l].d[j] + 2, 0.0);
  auto cl_ibar_at = [&](int64_t l, int e, int j, int64_t m) -> double {
    if (m > n_steps) return 0.0;
    return cl_ibar[6 * l + 3 * e + j][m % (sim.cl[l].d[j] + 2)];
  };
  auto V = [&](const double* vn, int32_t x) { return x >= 0 ? vn[x] : (x == -1 ? 0.0 : vs[-2 - x]); };
  for (int64_t n = n_steps; n >= 1; --n) {
    const double* vn = tape.data() + (size_t)(n - 1) * nn;
    const double* tg = v_target + (size_t)(n - 1) * nn;
    const double t = (double)n * net->dt;
    for (int64_t s = 0; s < ns; ++s)
      vs[s] = net->src_amp[s] * std::sin(2.0 * kPi * net->src_freq[s] * t + net->src_phase[s]);
    for (int64_t k = 0; k < nn; ++k) vbar[k] = 2.0 * (vn[k] - tg[k]);
    for (int64_t b = 0; b < nb; ++b) {
      if (net->br_kind[b] == 0) continue;
      double E = (net->br_kind[b] == 1 ? 2.0 : -2.0) * sim.g[b];
      if (net->br_k[b] >= 0) vbar[net->br_k[b]] += E * hbar[b];
      if (net->br_m[b] >= 0) vbar[net->br_m[b]] -= E * hbar[b];
    }
    for (int64_t l = 0; l < nl; ++l) {
      int64_t d = net->ln_d[l], d1 = d + 1;
      double y2 = 2.0 / net->ln_zc[l];
      vbar[net->ln_k[l]] += -y2 * ibar_m[l][(n + d) % d1];
      vbar[net->ln_m[l]] += -y2 * ibar_k[l][(n + d) % d1];
    }
    // coupled lines: c_e,j(n) = -(2/Z_j) (T_v^-1 v_e)_j - I_e,j(n) feeds the far
    // end's histories at n + d and n + d + 1
    for (int64_t l = 0; l < ncl; ++l) {
      const auto& L = sim.cl[l];
      for (int e = 0; e < 2; ++e) {
        const int32_t* nd = (e == 0 ? net->cl_k : net->cl_m) + 3 * l;
        for (int j = 0; j < 3; ++j) {
          const double x = (1.0 - L.f[j]) * cl_ibar_at(l, 1 - e, j, n + L.d[j]) +
                           L.f[j] * cl_ibar_at(l, 1 - e, j, n + L.d[j] + 1);
          cl_x[6 * l + 3 * e + j] = x;
          for (int p = 0; p < 3; ++p) vbar[nd[p]] += -L.y2[j] * L.tinv[3 * j + p] * x;
        }
      }
    }
    // w_n = G_n^{-T} vbar_n, per subsystem with the factors of step n
    for (int64_t w = 0; w < nr; ++w) sim.rs_on[w] = rs_tape[(size_t)(n - 1) * nr + w];
    for (int s = 0; s < sim.n_sub; ++s) {
      if (!sim.refactor_if_needed(s, n)) return -2;
      int m = (int)sim.nodes[s].size();
      std::vector<double> x(m);
      for (int i = 0; i < m; ++i) x[i] = vbar[sim.nodes[s][i]];
      lu_solve_transposed(m, sim.lu[s], sim.piv[s], x.data());
      for (int i = 0; i < m; ++i) w[sim.nodes[s][i]] = x[i];
    }
    for (int64_t b = 0; b < nb; ++b) {
      int32_t k = net->br_k[b], m = net->br_m[b];
      double aw = (k >= 0 ? w[k] : 0.0) - (m >= 0 ? w[m] : 0.0);
      double vb = V(vn, k) - V(vn, m);
      dg[b] += -aw * vb;
      double E = 0.0;
      if (net->br_kind[b] != 0) {
        E = (net->br_kind[b] == 1 ? 2.0 : -2.0) * sim.g[b];
        dg[b] += hbar[b] * (net->br_kind[b] == 1 ? 2.0 : -2.0) * vb;
      }
      // source amplitude terms
      if (k <= -2 || m <= -2) {
        int64_t s = k <= -2 ? (-2 - k) : (-2 - m);
        int32_t u = k <= -2 ? m : k;
        double dv = sim.g[b] * (u >= 0 ? w[u] : 0.0);
        if (net->br_kind[b] != 0) dv += (k <= -2 ? E : -E) * hbar[b];
        dA[s] += std::sin(2.0 * kPi * net->src_freq[s] * t + net->src_phase[s]) * dv;
      }
    }
    for (int64_t b = 0; b < nb; ++b) {
      if (net->br_kind[b] == 0) continue;
      int32_t k = net->br_k[b], m = net->br_m[b];
      double aw = (k >= 0 ? w[k] : 0.0) - (m >= 0 ? w[m] : 0.0);
      hbar[b] = (net->br_kind[b] == 1 ? 1.0 : -1.0) * hbar[b] - aw;
    }
    for (int64_t l = 0; l < nl; ++l) {
      int64_t d = net->ln_d[l], d1 = d + 1;
      double far_m = ibar_m[l][(n + d) % d1], far_k = ibar_k[l][(n + d) % d1];
      ibar_k[l][n % d1] = -w[net->ln_k[l]] - far_m;
      ibar_m[l][n % d1] = -w[net->ln_m[l]] - far_k;
    }
    // coupled lines: I_e,j(n) leaves the phase nodes through T_i and enters c_e,j(n)
    for (int64_t l = 0; l < ncl; ++l) {
      const auto& L = sim.cl[l];
      for (int e = 0; e < 2; ++e) {
        const int32_t* nd = (e == 0 ? net->cl_k : net->cl_m) + 3 * l;
        for (int j = 0; j < 3; ++j) {
          double tw = 0.0;
          for (int p = 0; p < 3; ++p) tw += L.ti[3 * p + j] * w[nd[p]];
          cl_ibar[6 * l + 3 * e + j][n % (L.d[j] + 2)] = -tw - cl_x[6 * l + 3 * e + j];
        }
      }
    }
  }
  for (int64_t b = 0; b < nb; ++b) {
    double x = net->br_val[b];
    double dgdp = net->br_kind[b] == 0 ? -1.0 / (x * x) : (net->br_kind[b] == 1 ? -net->dt / (2.0 * x * x) : 2.0 / net->dt);
    grad[b] = dg[b] * dgdp;
  }
  for (int64_t s = 0; s < ns; ++s) grad[nb + s] = dA[s];
  return 0;
}

extern "C" int orc_controls(const orc_net* net, int64_t n_steps, double* y_out) {
  if (!valid(net) || n_steps < 0 || (n_steps > 0 && net->n_cb > 0 && !y_out)) return -1;
  Sim<double> sim;
  sim.net = net;
  if (!sim.init(net->br_val, net->src_amp, false)) return -1;
  for (int64_t n = 1; n <= n_steps; ++n) {
    if (!sim.step(n)) return -2;
    for (int64_t b = 0; b < net->n_cb; ++b) y_out[(size_t)(n - 1) * net->n_cb + b] = sim.cy[b];
  }
  return 0;
}

extern "C" int orc_rs_states(const orc_net* net, int64_t n_steps, uint8_t* states) {
  if (!valid(net) || n_steps < 0 || (n_steps > 0 && net->n_rs > 0 && !states)) return -1;
  Sim<double> sim;
  sim.net = net;
  if (!sim.init(net->br_val, net->src_amp, false)) return -1;
  for (int64_t n = 1; n <= n_steps; ++n) {
    for (int64_t w = 0; w < net->n_rs; ++w) states[(size_t)(n - 1) * net->n_rs + w] = (uint8_t)sim.rs_on[w];
    if (!sim.step(n)) return -2;
  }
  return 0;
}

extern "C" int orc_partition(const orc_net* net, int32_t* sub_of_node, int64_t* n_sub) {
  if (!valid(net)) return -1;
  std::vector<int> sub;
  int ns = 0;
  components(net, sub, ns);
  for (int64_t i = 0; i < net->n_nodes; ++i) sub_of_node[i] = sub[i];
  *n_sub = ns;
  return 0;
}

extern "C" int orc_lu_solve(int64_t n, const double* A, const double* b, double* x) {
  if (n <= 0) return -1;
  std::vector<double> a(A, A + n * n);
  std::vector<int> piv;
  if (!lu_factor<double>((int)n, a, piv)) return -2;
  for (int64_t i = 0; i < n; ++i) x[i] = b[i];
  lu_solve<double>((int)n, a, piv, x);
  return 0;
}

// ---------------------------------------------------------------- sessions
//
// A session runs the loop window by window on a chosen set of subsystems.
// Subsystems meet only through lines, and a line end consumes at step n
// what the far end sent at step n - d (Sec. II-B: the travel time
// decouples the two ends), so a part of the network can run a window of
// up to d steps alone when the values its ends consume come in from
// wherever the far ends run.  The session exposes those sent values per
// line end for that exchange.  The other subsystems' processes 3 and 4 do
// not run; their node voltages stay 0, and what their ends send is wrong
// until the exchange overwrites it.

struct orc_session {
  const orc_net* net;
  Sim<double> sim;
  std::vector<double> br_value;
  int64_t n = 0;   // last completed step
};

namespace {

int64_t n_line_ends(const orc_net* net) { return 2 * net->n_ln + 6 * net->n_cl + 2 * net->n_fl; }

// The storage of the value line end x sent at step m (which must still be
// held: m within the last d + 1 steps), or nullptr for an unknown end.
double* sent_slot(orc_session* S, int64_t x, int64_t m) {
  const orc_net* net = S->net;
  Sim<double>& sim = S->sim;
  if (x < 0) return nullptr;
  if (x < 2 * net->n_ln) {   // end k's value waits in end m's ring, and vice versa, at the slot of step m + d
    const int64_t l = x / 2, d1 = net->ln_d[l] + 1;
    auto& ring = (x % 2 == 0) ? sim.ring_m[l] : sim.ring_k[l];
    return &ring[(m + net->ln_d[l]) % d1];
  }
  x -= 2 * net->n_ln;
  if (x < 6 * net->n_cl) {   // coupled line l, end e, mode j: by sending step
    const int64_t l = x / 6;
    const int e = (int)((x % 6) / 3), j = (int)(x % 3);
    auto& L = sim.cl[l];
    return &L.c[e][j][m % (L.d[j] + 2)];
  }
  x -= 6 * net->n_cl;
  if (x < 2 * net->n_fl) {   // frequency-dependent line l, end e: by sending step
    auto& L = sim.fl[x / 2];
    return &L.w[x % 2][m % (L.d + 3)];
  }
  return nullptr;
}

int64_t end_delay(const orc_net* net, const Sim<double>& sim, int64_t x) {
  if (x < 2 * net->n_ln) return net->ln_d[x / 2];
  x -= 2 * net->n_ln;
  if (x < 6 * net->n_cl) return sim.cl[x / 6].d[x % 3];
  x -= 6 * net->n_cl;
  return sim.fl[x / 2].d;
}

}  // namespace

extern "C" orc_session* orc_open(const orc_net* net) {
  if (!valid(net)) return nullptr;
  orc_session* S = new orc_session;
  S->net = net;
  S->br_value.assign(net->br_val, net->br_val + net->n_br);
  S->sim.net = net;
  if (!S->sim.init(S->br_value.data(), net->src_amp, false)) {
    delete S;
    return nullptr;
  }
  return S;
}

extern "C" int orc_advance(orc_session* S, int64_t n_steps, const uint8_t* active, double* v_out) {
  if (!S || n_steps < 0) return -1;
  Sim<double>& sim = S->sim;
  if (active != nullptr && S->net->n_cb > 0) return -1;   // control blocks may join subsystems without a line
  sim.active.clear();
  if (active != nullptr)
    for (int s = 0; s < sim.n_sub; ++s) sim.active.push_back(active[s] ? 1 : 0);
  for (int64_t k = 0; k < n_steps; ++k) {
    if (!sim.step(S->n + 1)) return -2;
    ++S->n;
    if (v_out)
      for (int64_t i = 0; i < S->net->n_nodes; ++i) v_out[k * S->net->n_nodes + i] = sim.v[i];
  }
  return 0;
}

extern "C" int orc_line_ends(const orc_net* net, int32_t* node, int32_t* far, int32_t* d) {
  if (!valid(net)) return -1;
  int64_t x = 0;
  for (int64_t l = 0; l < net->n_ln; ++l, x += 2) {
    node[x] = net->ln_k[l];
    node[x + 1] = net->ln_m[l];
    far[x] = (int32_t)(x + 1);
    far[x + 1] = (int32_t)x;
    d[x] = d[x + 1] = net->ln_d[l];
  }
  for (int64_t l = 0; l < net->n_cl; ++l)
    for (int e = 0; e < 2; ++e)
      for (int j = 0; j < 3; ++j, ++x) {
        node[x] = (e == 0 ? net->cl_k : net->cl_m)[3 * l];
        far[x] = (int32_t)(x + (e == 0 ? 3 : -3));
        d[x] = (int32_t)std::floor(net->cl_tau[3 * l + j] / net->dt);
      }
  for (int64_t l = 0; l < net->n_fl; ++l, x += 2) {
    node[x] = net->fl_k[l];
    node[x + 1] = net->fl_m[l];
    far[x] = (int32_t)(x + 1);
    far[x + 1] = (int32_t)x;
    d[x] = d[x + 1] = (int32_t)std::floor(net->fl_tau[l] / net->dt);
  }
  return 0;
}

extern "C" int orc_sent(orc_session* S, int64_t end, int64_t n0, int64_t w, double* vals, int set) {
  if (!S || end < 0 || end >= n_line_ends(S->net) || w < 0) return -1;
  const int64_t d = end_delay(S->net, S->sim, end);
  // only the last d + 1 steps' values are still held
  if (n0 < 1 || n0 + w - 1 > S->n || n0 <= S->n - (d + 1)) return -1;
  for (int64_t j = 0; j < w; ++j) {
    double* p = sent_slot(S, end, n0 + j);
    if (set) *p = vals[j];
    else vals[j] = *p;
  }
  return 0;
}

extern "C" void orc_close(orc_session* S) { delete S; }

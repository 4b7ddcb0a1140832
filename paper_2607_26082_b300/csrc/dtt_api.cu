// Host side of libdtt: the C ABI of include/dtt.h.
//
// A dtt_grid owns every device buffer of one cell.  dtt_solve_step runs Algorithm 1 (or
// one increment of Algorithm 2) as a fixed sequence of kernel launches per iteration,
// captured once into a CUDA graph of `graph_iters` iterations and replayed until the
// device-side control block reports convergence, the iteration cap or divergence; the
// host only reads a few bytes of that block between graph launches.
#include "dtt.h"
#include "dtt_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace dtt;

namespace {

thread_local std::string g_err;

dtt_status fail(dtt_status s, const std::string& m) {
  g_err = m;
  return s;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(DTT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKL(rc)                                                                             \
  do {                                                                                      \
    int r_ = (rc);                                                                          \
    if (r_ != 0) return fail(DTT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)r_)); \
  } while (0)

template <typename P>
dtt_status dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return DTT_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? DTT_ERR_OOM : DTT_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return DTT_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

}  // namespace

#include "grid_internal.cuh"

dtt_status dtt::set_error(dtt_status s, const std::string& msg) { return fail(s, msg); }

namespace {

const int kIP[2] = {2, 1};

void invalidate_graph(dtt_grid* G) {
  G->version += 1;
  if (G->gexec) cudaGraphExecDestroy(G->gexec);
  G->gexec = nullptr;
  G->g_key = -1;
}

int ttype(int b0, int b1) {
  if (b0 == BC_P || b1 == BC_P) return (b0 == BC_P && b1 == BC_P) ? T_DHT : -1;
  if (b0 == BC_N && b1 == BC_N) return T_DCT1;
  if (b0 == BC_N && b1 == BC_D) return T_DCT3;
  if (b0 == BC_D && b1 == BC_D) return T_DST1;
  return T_DST3;  // D, N
}

// Transform matrices of one axis: F (spectral k, node j) and B (node j, spectral k), both
// nn x nn with zero rows/columns outside the selection (Section 3.2.2, Table 3), plus
// sin^2(q_k / 2) at every spectral position (0 where unused).
void build_axis(int type, int n, int nn, std::vector<double>& F, std::vector<double>& B, std::vector<double>& cq,
                std::vector<double>& cc) {
  F.assign((size_t)nn * nn, 0.0);
  B.assign((size_t)nn * nn, 0.0);
  cq.assign(nn, 0.0);
  cc.assign(nn, 1.0);
  const double pi = 3.14159265358979323846;
  switch (type) {
    case T_DCT1:
      for (int k = 0; k <= n; ++k) {
        cq[k] = std::pow(std::sin(0.5 * pi * k / n), 2);
        cc[k] = std::pow(std::cos(0.5 * pi * k / n), 2);
        for (int j = 0; j <= n; ++j) {
          double c = std::cos(pi * (double)j * k / n);
          double wj = (j == 0 || j == n) ? 0.5 : 1.0;
          double wk = (k == 0 || k == n) ? 0.5 : 1.0;
          F[(size_t)k * nn + j] = wj * c;
          B[(size_t)j * nn + k] = 2.0 / n * wk * c;
        }
      }
      break;
    case T_DCT3:
      for (int k = 0; k < n; ++k) {
        cq[k] = std::pow(std::sin(0.5 * pi * (2.0 * k + 1.0) / (2.0 * n)), 2);
        cc[k] = std::pow(std::cos(0.5 * pi * (2.0 * k + 1.0) / (2.0 * n)), 2);
        for (int j = 0; j < n; ++j) {
          double c = std::cos(pi * j * (2.0 * k + 1.0) / (2.0 * n));
          F[(size_t)k * nn + j] = (j == 0 ? 0.5 : 1.0) * c;
          B[(size_t)j * nn + k] = 2.0 / n * c;
        }
      }
      break;
    case T_DST1:
      for (int k = 1; k < n; ++k) {
        cq[k] = std::pow(std::sin(0.5 * pi * k / n), 2);
        cc[k] = std::pow(std::cos(0.5 * pi * k / n), 2);
        for (int j = 1; j < n; ++j) {
          double sv = std::sin(pi * (double)j * k / n);
          F[(size_t)k * nn + j] = sv;
          B[(size_t)j * nn + k] = 2.0 / n * sv;
        }
      }
      break;
    case T_DST3:
      for (int k = 0; k < n; ++k) {
        cq[k] = std::pow(std::sin(0.5 * pi * (2.0 * k + 1.0) / (2.0 * n)), 2);
        cc[k] = std::pow(std::cos(0.5 * pi * (2.0 * k + 1.0) / (2.0 * n)), 2);
        for (int j = 1; j <= n; ++j) {
          double sv = std::sin(pi * j * (2.0 * k + 1.0) / (2.0 * n));
          F[(size_t)k * nn + j] = (j == n ? 0.5 : 1.0) * sv;
          B[(size_t)j * nn + k] = 2.0 / n * sv;
        }
      }
      break;
    case T_DHT:
      for (int k = 0; k < n; ++k) {
        cq[k] = std::pow(std::sin(pi * (double)k / n), 2);
        cc[k] = std::pow(std::cos(pi * (double)k / n), 2);
        for (int j = 0; j < n; ++j) {
          double th = 2.0 * pi * (double)((long long)j * k % n) / n;
          double cas = std::cos(th) + std::sin(th);
          F[(size_t)k * nn + j] = cas;
          B[(size_t)j * nn + k] = cas / n;
        }
      }
      break;
  }
}

// Tensor-core z pass: the active node rows and spectral positions of each component's z
// transform (Table 3), one operand size for the three components, and the forward and
// inverse matrices packed for the kernel.  Grids whose z operand exceeds 256 keep the
// FFT (or dense) z pass.  DTT_Z_TENSOR=1 in the environment selects the route at creation.
dtt_status build_tz(dtt_grid* G) {
  const int n = G->g.nvox[2], nn = G->g.nn[2];
  int P = 0;
  for (int c = 0; c < 3; ++c) {
    TzComp& t = G->tz[c];
    switch (G->types[c][2]) {
      case T_DCT1: t.j0 = 0; t.nj = n + 1; t.k0 = 0; t.nk = n + 1; break;
      case T_DCT3: t.j0 = 0; t.nj = n; t.k0 = 0; t.nk = n; break;
      case T_DST1: t.j0 = 1; t.nj = n - 1; t.k0 = 1; t.nk = n - 1; break;
      case T_DST3: t.j0 = 1; t.nj = n; t.k0 = 0; t.nk = n; break;
      default: t.j0 = 0; t.nj = n; t.k0 = 0; t.nk = n; break;   // Hartley (periodic)
    }
    P = std::max(P, std::max(t.nj, t.nk));
  }
  P = (P + 31) / 32 * 32;
  G->tz_ok = false;
  if (P > 256 || n < 2) return DTT_OK;
  for (int c = 0; c < 3; ++c) {
    TzComp& t = G->tz[c];
    t.P = P;
    std::vector<double> F, B, cq, cc;
    build_axis(G->types[c][2], n, nn, F, B, cq, cc);
    std::vector<float> pf, pi;
    tz_pack_matrix(F.data(), nn, t.k0, t.nk, t.j0, t.nj, P, pf);   // rows: spectral, columns: nodes
    tz_pack_matrix(B.data(), nn, t.j0, t.nj, t.k0, t.nk, P, pi);   // rows: nodes, columns: spectral
    dtt_status s = dalloc(&G->tz_mat[c], (pf.size() + pi.size()) * sizeof(float));
    if (s != DTT_OK) return s;
    CK(cudaMemcpy(G->tz_mat[c], pf.data(), pf.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->tz_mat[c] + pf.size(), pi.data(), pi.size() * 4, cudaMemcpyHostToDevice));
    t.fwd = G->tz_mat[c];
    t.inv = G->tz_mat[c] + pf.size();
  }
  if (!G->tz_err) {
    dtt_status s = dalloc(&G->tz_err, sizeof(unsigned int));
    if (s != DTT_OK) return s;
  }
  CK(cudaMemset(G->tz_err, 0, sizeof(unsigned int)));
  G->tz_ok = true;
  const char* e = std::getenv("DTT_Z_TENSOR");
  if (e && e[0] == '1') G->z_route = 1;
  return DTT_OK;
}

// 0 when no tensor-core z pass has recorded a timed-out wait, else DTT_ERR_CUDA.
dtt_status check_tz(dtt_grid* G) {
  if (!G->tz_err) return DTT_OK;
  unsigned int e = 0;
  CK(cudaMemcpy(&e, G->tz_err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e) {
    cudaMemset(G->tz_err, 0, sizeof(unsigned int));
    return fail(DTT_ERR_CUDA, "tensor-core z pass: a bounded wait ran out (the CTA skipped its work)");
  }
  return DTT_OK;
}

// FFT plan of one axis: length L = 2n (n on a periodic axis) factored into radices 4, 2
// and 3; axes whose length has another prime factor, or n < 4, keep the dense contraction.
dtt_status build_fft_axis(dtt_grid* G, int d) {
  FftAxisInfo& f = G->fft[d];
  f = FftAxisInfo{};
  const int n = G->g.nvox[d];
  const int L = G->g.periodic[d] ? n : 2 * n;
  if (n < 4 || std::getenv("DTT_DENSE_TRANSFORMS")) return DTT_OK;
  int m = L, ns = 0;
  int rad[12];
  while (m % 4 == 0 && ns < 12) { rad[ns++] = 4; m /= 4; }
  while (m % 2 == 0 && ns < 12) { rad[ns++] = 2; m /= 2; }
  while (m % 3 == 0 && ns < 12) { rad[ns++] = 3; m /= 3; }
  if (m != 1) return DTT_OK;
  const double pi = 3.14159265358979323846;
  const size_t csz = 2 * G->esz;
  std::vector<double> tw(2 * (size_t)L), ph(2 * (size_t)(2 * n));
  for (int q = 0; q < L; ++q) {
    tw[2 * q] = std::cos(2.0 * pi * q / L);
    tw[2 * q + 1] = -std::sin(2.0 * pi * q / L);
  }
  for (int j = 0; j < 2 * n; ++j) {
    ph[2 * j] = std::cos(pi * j / (2.0 * n));
    ph[2 * j + 1] = -std::sin(pi * j / (2.0 * n));
  }
  dtt_status s = dalloc(&G->fft_tw[d], (size_t)L * csz);
  if (s == DTT_OK) s = dalloc(&G->fft_ph[d], (size_t)(2 * n) * csz);
  if (s != DTT_OK) return s;
  if (G->esz == 8) {
    CK(cudaMemcpy(G->fft_tw[d], tw.data(), tw.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->fft_ph[d], ph.data(), ph.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> twf(tw.begin(), tw.end()), phf(ph.begin(), ph.end());
    CK(cudaMemcpy(G->fft_tw[d], twf.data(), twf.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->fft_ph[d], phf.data(), phf.size() * 4, cudaMemcpyHostToDevice));
  }
  f.use = 1;
  f.L = L;
  f.nst = ns;
  for (int q = 0; q < ns; ++q) f.radix[q] = rad[q];
  f.tw = G->fft_tw[d];
  f.ph = G->fft_ph[d];
  // stage-1 twiddles of the warp-register passes (mixed path, non-periodic, L = 32 R)
  const int R = wfft_radix(L);
  if (G->esz == 4 && !G->g.periodic[d] && R) {
    std::vector<float> t1(2 * (size_t)R * 32);
    for (int k1 = 0; k1 < R; ++k1)
      for (int l = 0; l < 32; ++l) {
        const int m = (l * k1) % L;
        t1[2 * (k1 * 32 + l)] = (float)std::cos(2.0 * pi * m / L);
        t1[2 * (k1 * 32 + l) + 1] = (float)-std::sin(2.0 * pi * m / L);
      }
    dtt_status s2 = dalloc(&G->fft_tw1[d], t1.size() * 4);
    if (s2 != DTT_OK) return s2;
    CK(cudaMemcpy(G->fft_tw1[d], t1.data(), t1.size() * 4, cudaMemcpyHostToDevice));
    f.tw1 = G->fft_tw1[d];
  }
  return DTT_OK;
}

bool comp_has_null(const dtt_grid* G, int c) {
  bool all0 = true;
  int npi = 0;
  for (int d = 0; d < 3; ++d) {
    int t = G->types[c][d];
    bool q0 = (t == T_DCT1 || t == T_DHT);
    bool qpi = (t == T_DCT1) || (t == T_DHT && G->g.nvox[d] % 2 == 0);
    all0 = all0 && q0;
    npi += qpi ? 1 : 0;
  }
  if (all0) return true;
  if (G->g.scheme == SCHEME_TETRA2) return npi == 3;
  return npi >= 2;
}

// W_c and DOF flag of node n (host).
void host_node_W(const dtt_grid* G, int c, long long n, bool& dof, double& W) {
  int idx[3];
  idx[0] = (int)(n % G->g.nn[0]);
  long long r = n / G->g.nn[0];
  idx[1] = (int)(r % G->g.nn[1]);
  idx[2] = (int)(r / G->g.nn[1]);
  dof = true;
  W = 1.0;
  for (int d = 0; d < 3; ++d) {
    if (G->g.periodic[d]) continue;
    int f = -1;
    if (idx[d] == 0) f = 0;
    else if (idx[d] == G->g.nn[d] - 1) f = 1;
    if (f < 0) continue;
    int t = G->g.bc[d][f][c];
    if (t == BC_D) dof = false;
    else if (t == BC_N) W *= 0.5;
  }
}

double host_ustar(const dtt_grid* G, int c, long long n) {
  double X[3];
  X[0] = G->g.h * (double)(n % G->g.nn[0]);
  long long r = n / G->g.nn[0];
  X[1] = G->g.h * (double)(r % G->g.nn[1]);
  X[2] = G->g.h * (double)(r / G->g.nn[1]);
  return G->eps[c][0] * X[0] + G->eps[c][1] * X[1] + G->eps[c][2] * X[2];
}

// Per xy tile of the mixed residual kernel, the z range of the nodes where the projections
// correct u~ (row DOFs and contact-face nodes) and whose correction reaches the tile's
// nodes through A0's one-node stencil: a node at (i, j, k) marks the tiles whose node halo
// (one node around the owned block) contains (i, j), with k; a periodic axis wraps.
dtt_status build_tile_z(dtt_grid* G, const std::vector<long long>& marked) {
  const int tx = residual_f32_tile(0), ty = residual_f32_tile(1);
  const int nnx = G->g.nn[0], nny = G->g.nn[1], nnz = G->g.nn[2];
  const int ntx = res_ntx(G->g, tx), nty = (nny + ty - 1) / ty;
  std::vector<int2> t((size_t)ntx * nty, make_int2(INT32_MAX, INT32_MIN));
  for (long long n : marked) {
    const int i = (int)(n % nnx), j = (int)((n / nnx) % nny), k = (int)(n / ((long long)nnx * nny));
    int zlo = k, zhi = k;
    if (G->g.periodic[2] && (k == 0 || k == nnz - 1)) {
      zlo = -1;
      zhi = nnz;
    }
    for (int di = -1; di <= 1; ++di) {
      int ii = i + di;
      if (G->g.periodic[0]) ii = (ii + nnx) % nnx;
      if (ii < 0 || ii >= nnx) continue;
      for (int dj = -1; dj <= 1; ++dj) {
        int jj = j + dj;
        if (G->g.periodic[1]) jj = (jj + nny) % nny;
        if (jj < 0 || jj >= nny) continue;
        int2& r = t[(size_t)(jj / ty) * ntx + res_tile_of_x(G->g, ii, tx)];
        r.x = std::min(r.x, zlo);
        r.y = std::max(r.y, zhi);
      }
    }
  }
  // the exact mode's residual runs as a flux-free pass plus one CTA per marked tile over
  // its marked planes +- 1 when those ranges are short (else one pass does everything)
  int span = 0;
  for (const int2& r : t)
    if (r.x <= r.y) span = std::max(span, r.y - r.x + 3);
  const int split = span == 0 ? 2 : (span <= 16 ? 1 : 0);
  if (split != G->res_split) {
    G->res_split = split;
    invalidate_graph(G);
  }
  if (G->tile_cap < (int)t.size()) {
    dfree(G->d_tile_z);
    G->tile_cap = 0;
    dtt_status s = dalloc(&G->d_tile_z, t.size() * sizeof(int2));
    if (s != DTT_OK) return s;
    G->tile_cap = (int)t.size();
  }
  CK(cudaMemcpy(G->d_tile_z, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice));
  return DTT_OK;
}

dtt_status rebuild_cmask(dtt_grid* G) {
  std::vector<uint8_t> m((size_t)G->NN, 0);
  std::vector<long long> marked;
  for (size_t e = 0; e < G->h_dof.size(); ++e) {
    long long d = G->h_dof[e];
    int c = (int)(d / G->NN);
    m[(size_t)(d - c * G->NN)] |= (uint8_t)(1u << c);
    marked.push_back(d - c * G->NN);
  }
  if (G->contact) {
    std::vector<long long> nodes(G->nface);
    CK(cudaMemcpy(nodes.data(), G->d_face, sizeof(long long) * G->nface, cudaMemcpyDeviceToHost));
    for (long long n : nodes) {
      m[(size_t)n] |= 7u;
      marked.push_back(n);
    }
  }
  CK(cudaMemcpy(G->cmask, m.data(), (size_t)G->NN, cudaMemcpyHostToDevice));
  return build_tile_z(G, marked);
}

// Exact residual mode of the mixed path (ResidualArgs::exact): valid when the Green step
// inverts the Paux A0 on every mode, i.e. no component has null modes.
bool exact_residual(const dtt_grid* G) {
  if (G->prec != DTT_PREC_MIXED || G->g.ref_iso || !G->exact_ok || !G->d_tile_z) return false;
  for (int c = 0; c < 3; ++c)
    if (comp_has_null(G, c)) return false;
  return true;
}

int res_blocks(const dtt_grid* G) {
  return G->prec == DTT_PREC_FP64 ? residual_nblocks<double>(G->g) : residual_nblocks<float>(G->g);
}

dtt_status ensure_partials(dtt_grid* G) {
  size_t need = RES_STRIDE * (size_t)std::max(residual_blocks(G->g), residual_f32_blocks(G->g)) +
                PROJ_STRIDE * ((size_t)(G->nrows + 255) / 256 + 1) + CONT_STRIDE * ((size_t)contact_blocks(G->nface) + 1) +
                4 * (size_t)acv_blocks(G->g) + 64;
  if (need <= G->part_cap) return DTT_OK;
  dfree(G->d_part);
  dtt_status s = dalloc(&G->d_part, need * sizeof(double));
  if (s != DTT_OK) return s;
  G->part_cap = need;
  return DTT_OK;
}

struct PartRegions {
  double *res, *proj, *cont, *acv;
  int nres, nproj, ncont, nacv;
};

PartRegions regions(dtt_grid* G) {
  PartRegions r;
  r.nres = res_blocks(G);
  r.nproj = (G->nrows + 255) / 256;
  r.ncont = G->contact ? contact_blocks(G->nface) : 0;
  r.nacv = acv_blocks(G->g);
  r.res = G->d_part;
  r.proj = r.res + RES_STRIDE * r.nres;
  r.cont = r.proj + PROJ_STRIDE * (r.nproj + 1);
  r.acv = r.cont + CONT_STRIDE * (r.ncont + 1);
  return r;
}

RowsDev rows_dev(dtt_grid* G) {
  RowsDev r;
  r.nrows = G->nrows;
  r.ptr = G->d_ptr;
  r.dof = G->d_dof;
  r.a = G->d_a;
  r.b = G->d_b;
  r.target = G->d_target;
  r.mult = G->d_mult;
  r.ab = G->d_ab;
  r.aa = G->d_aa;
  return r;
}

ContactArgs contact_args(dtt_grid* G, double* cont_part) {
  ContactArgs a{};
  a.g = G->g;
  a.c.nnodes_face = G->nface;
  a.c.node = G->d_face;
  a.c.active = G->d_active;
  a.c.vgap = G->d_vgap;
  a.c.vreact = G->d_vreact;
  a.c.vgap_prev = G->d_vgap_prev;
  a.c.vreact_prev = G->d_vreact_prev;
  a.c.gap = G->d_gap;
  a.c.fn = G->d_fn;
  a.c.nvec = G->d_nvec;
  for (int c = 0; c < 3; ++c) a.c.center[c] = G->center[c];
  a.c.radius = G->radius;
  a.u64 = G->u64;
  a.uhi = G->uhi;
  a.ulo = G->ulo;
  std::memcpy(a.eps, G->eps, sizeof(a.eps));
  a.ctrl = G->d_ctrl;
  a.partials = cont_part;
  return a;
}

TransformTables tables(dtt_grid* G) {
  TransformTables t;
  for (int d = 0; d < 3; ++d) t.fft[d] = G->fft[d];
  t.tz_use = (G->z_route == 1 && G->tz_ok && G->prec == DTT_PREC_MIXED && !G->g.ref_iso) ? 1 : 0;
  for (int c = 0; c < 3; ++c) t.tz[c] = G->tz[c];
  t.tz_err = G->tz_err;
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) t.types[c][d] = G->types[c][d];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      t.fwd[c][d] = G->fwd[c][d];
      t.inv[c][d] = G->inv[c][d];
      t.sin2q[c][d] = G->sin2q[c][d];
      t.cos2q[c][d] = G->cos2q[c][d];
      t.sin2q_f[c][d] = G->sin2q_f[c][d];
      t.cos2q_f[c][d] = G->cos2q_f[c][d];
    }
  t.lam0 = G->lam0;
  t.mu0 = G->mu0;
  // Null modes: a_c vanishes exactly (up to rounding) there; every other spectral point
  // has a_c >= ~mu0 (pi / 2n)^2 / h^2.  Threshold: 1e-12 x an upper bound of a_c
  // ((lambda0 + 6 mu0) * 4 / h^2, since every S_j <= 4 / h^2).
  double bound = (G->lam0 + 6.0 * G->mu0) * 4.0 / (G->g.h * G->g.h);
  for (int c = 0; c < 3; ++c) t.null_thr[c] = 1e-12 * bound;
  for (int d = 0; d < 3; ++d) {
    t.iso.s[d] = G->iso_s[d];
    t.iso.c[d] = G->iso_c[d];
    t.iso.sf[d] = G->iso_sf[d];
    t.iso.cf[d] = G->iso_cf[d];
    t.iso.valid[d] = G->iso_valid[d];
    t.iso.sign[d] = (G->types[d][d] == T_DST1 || G->types[d][d] == T_DST3) ? 1 : -1;
  }
  t.iso.null_thr = 1e-12 * bound;
  return t;
}

// Optional per-group event marks (dtt_profile_iteration); null when not profiling.
cudaEvent_t* g_prof_ev = nullptr;
inline void prof_mark(int k, cudaStream_t s) {
  if (g_prof_ev) cudaEventRecord(g_prof_ev[k], s);
}

// Green step (forward DT, Green multiply, inverse DT) of `in` (or of the ring slot
// i % 4 when in_ring is given); the result lands in out, or, with `increment`, is added to
// u~ and stored as the step.  When the z axis takes the FFT route, the forward z transform,
// the Green multiply and the inverse z transform run as one fused pass; when the x axis
// takes it too, the increment is fused into the inverse x pass.
template <typename T>
dtt_status enqueue_green(dtt_grid* G, const T* in, void* const* in_ring, T* out, T* tmp, bool increment,
                         const Ctrl* ctrl, int comp0, int ncomp, bool no_step = false) {
  TransformTables tt = tables(G);
  cudaStream_t s = G->stream;
  // mixed path: five warp-register sweeps, each reading contiguous rows (k_wfft.cu)
  if constexpr (sizeof(T) == 4) {
    if (G->fft_warp && !tt.tz_use && !G->g.fft_generic && wfft_supported(G->g, tt)) {
      const bool alias = (in_ring == nullptr && (const void*)in == (const void*)out);
      T* b1 = alias ? tmp : out;
      T* b2 = alias ? out : tmp;
      IncrTarget it{G->u64, G->uhi, G->ulo, no_step ? nullptr : G->step};
      CKL(launch_wfft_green(G->g, tt, in, in_ring, b1, b2, out, increment ? &it : nullptr, comp0, ncomp, ctrl, s,
                            g_prof_ev ? prof_mark : nullptr));
      return DTT_OK;
    }
  }
  // the isotropic medium couples the components: its Green step needs all three spectra,
  // so it takes the unfused route
  if ((tt.fft[2].use || tt.tz_use) && !G->g.ref_iso) {
    const bool alias = (in_ring == nullptr && (const void*)in == (const void*)out);
    T* b1 = alias ? tmp : out;
    T* b2 = alias ? out : tmp;
    CKL(launch_transform_axis<T>(G->g, in, b1, tt, 0, 0, comp0, ncomp, ctrl, s, in_ring));
    CKL(launch_transform_axis<T>(G->g, b1, b2, tt, 1, 0, comp0, ncomp, ctrl, s));
    prof_mark(4, s);
    CKL(launch_z_green<T>(G->g, b2, b1, tt, comp0, ncomp, ctrl, s));
    prof_mark(5, s);
    CKL(launch_transform_axis<T>(G->g, b1, b2, tt, 1, 1, comp0, ncomp, ctrl, s));
    if (increment && tt.fft[0].use) {
      IncrTarget it{G->u64, G->uhi, G->ulo, no_step ? nullptr : G->step};
      CKL(launch_transform_axis<T>(G->g, b2, b1, tt, 0, 1, comp0, ncomp, ctrl, s, nullptr, &it));
      prof_mark(6, s);
      return DTT_OK;
    }
    CKL(launch_transform_axis<T>(G->g, b2, b1, tt, 0, 1, comp0, ncomp, ctrl, s));
    prof_mark(6, s);
    if (increment) {
      CKL(launch_add_increment<T>(G->g, b1, G->u64, G->uhi, G->ulo, no_step ? nullptr : (T*)G->step, ctrl, s));
    } else if (b1 != out) {
      CK(cudaMemcpyAsync(out, b1, (size_t)3 * G->NN * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    return DTT_OK;
  }
  CKL(launch_transform_axis<T>(G->g, in, tmp, tt, 0, 0, comp0, ncomp, ctrl, s, in_ring));
  CKL(launch_transform_axis<T>(G->g, tmp, out, tt, 1, 0, comp0, ncomp, ctrl, s));
  CKL(launch_transform_axis<T>(G->g, out, tmp, tt, 2, 0, comp0, ncomp, ctrl, s));
  prof_mark(4, s);
  if (G->g.ref_iso) CKL(launch_green_iso<T>(G->g, tmp, tt, ctrl, s));
  else CKL(launch_green_multiply<T>(G->g, tmp, tt, G->g.scheme, ctrl, s));
  prof_mark(5, s);
  CKL(launch_transform_axis<T>(G->g, tmp, out, tt, 2, 1, comp0, ncomp, ctrl, s));
  CKL(launch_transform_axis<T>(G->g, out, tmp, tt, 1, 1, comp0, ncomp, ctrl, s));
  CKL(launch_transform_axis<T>(G->g, tmp, out, tt, 0, 1, comp0, ncomp, ctrl, s));
  prof_mark(6, s);
  if (increment) CKL(launch_add_increment<T>(G->g, out, G->u64, G->uhi, G->ulo, no_step ? nullptr : (T*)G->step, ctrl, s));
  return DTT_OK;
}

// One iteration of Algorithm 1 / Algorithm 2 as a fixed launch sequence.
//   ACV on p~ (difference form): residual (p_i, R_{i-1}) -> proj_P -> contact -> control ->
//     Gram row -> alpha -> Green input g_i -> Green step (u~ += G g_i, step) -> proj_U.
//   ACV on u~ (FP64): R_{i-1} = u~_i - S_{i-1}, alpha, u~ <- combination, S_i = u~, then
//     residual (p_i) -> ... -> Green step on p_i.
template <typename T>
dtt_status enqueue_iteration(dtt_grid* G, int acv_on, bool acv) {
  cudaStream_t s = G->stream;
  PartRegions pr = regions(G);
  Ctrl* ctrl = G->d_ctrl;
  const bool diff = acv && acv_on == DTT_ACV_P;
  prof_mark(0, s);
  if (acv && acv_on == DTT_ACV_U) {
    CKL(launch_acv_store<T>(G->g, 0, G->d_Sring, G->d_Rring, G->u64, pr.acv, ctrl, s));
    CKL(launch_ctrl_acv(ctrl, pr.acv, pr.nacv, s));
    CKL(launch_acv_accel<T>(G->g, 0, G->d_Sring, G->d_Rring, (T*)G->gbuf, G->u64, ctrl, s));
  }
  ResidualArgs ra{};
  ra.g = G->g;
  ra.u64 = G->u64;
  ra.uhi = G->uhi;
  ra.ulo = G->ulo;
  ra.phase = G->phase;
  ra.lam = G->d_lam;
  ra.mu = G->d_mu;
  ra.nphase = G->nphase;
  ra.cmask = G->cmask;
  std::memcpy(ra.eps, G->eps, sizeof(ra.eps));
  ra.lam0 = G->lam0;
  ra.mu0 = G->mu0;
  ra.mode = diff ? 1 : 2;
  ra.pout = G->gbuf;
  ra.dfield = G->step;
  const bool exact = sizeof(T) == 4 && diff && exact_residual(G);
  ra.exact = exact ? 1 : 0;
  ra.tile_z = G->d_tile_z;
  ra.split = exact ? G->res_split : 0;
  for (int k = 0; k < 4; ++k) {
    ra.pring[k] = G->S[k];
    ra.gring[k] = G->Gr[k];
    ra.rring[k] = G->R[k];
  }
  ra.partials = pr.res;
  ra.ctrl = ctrl;
  CKL(launch_residual<T>(ra, s));
  prof_mark(1, s);
  const int rm = diff ? 1 : 0;
  const int fused = (diff && sizeof(T) == 4) ? 1 : 0;   // the FP32 residual kernel fuses the Gram row
  if (G->nrows > 0)
    CKL(launch_proj_P_rows<T>(G->g, rows_dev(G), (T*)G->gbuf, G->d_Sring, G->d_Rring, rm, fused, pr.proj, ctrl, s,
                              exact ? (T*)G->step : nullptr));
  ContactArgs ca = contact_args(G, pr.cont);
  ca.step_clear = exact ? G->step : nullptr;
  if (G->contact) CKL(launch_contact_eval<T>(ca, (T*)G->gbuf, G->d_Sring, G->d_Rring, rm, fused, s));
  // residual control and (no contact, Gram row fused into the residual and projection
  // kernels) the Anderson solve in one launch
  const bool merged = diff && fused && !G->contact;
  if (merged) {
    CKL(launch_ctrl_residual_acv(ctrl, pr.res, pr.nres, pr.proj, G->nrows > 0 ? pr.nproj : 0, G->g.h, G->NN, G->NV,
                                 s));
  } else {
    CKL(launch_ctrl_residual(ctrl, pr.res, pr.nres, pr.proj, G->nrows > 0 ? pr.nproj : 0, pr.cont, pr.ncont, G->g.h,
                             G->NN, G->NV, s));
  }
  if (G->contact) {
    CKL(launch_contact_update(ca, s));
    CKL(launch_ctrl_contact(ctrl, s));
  }
  prof_mark(2, s);
  if (diff) {
    if (fused) {
      if (!merged)
        CKL(launch_ctrl_acv_fused(ctrl, pr.res, pr.nres, pr.proj, G->nrows > 0 ? pr.nproj : 0, pr.cont, pr.ncont, s));
    } else {
      CKL(launch_acv_gram<T>(G->g, G->d_Rring, pr.acv, ctrl, s));
      CKL(launch_ctrl_acv(ctrl, pr.acv, pr.nacv, s));
    }
    CKL(launch_acv_green_input<T>(G->g, G->d_Sring, G->d_Gring, G->d_Gown, G->d_Rring, ctrl, exact ? 1 : 0,
                                  G->d_tile_z, s));
  }
  prof_mark(3, s);
  dtt_status st = diff ? enqueue_green<T>(G, nullptr, G->d_Gring, (T*)G->spec2, (T*)G->spec, true, ctrl, 0, 3, exact)
                       : enqueue_green<T>(G, (const T*)G->gbuf, nullptr, (T*)G->spec2, (T*)G->spec, true, ctrl, 0, 3);
  if (st != DTT_OK) return st;
  prof_mark(7, s);
  if (G->nrows > 0 && !G->contact) {
    // the rows' projection is the last step: its last CTA ends the iteration
    CKL(launch_proj_U_rows_end<T>(G->g, rows_dev(G), G->u64, G->uhi, G->ulo, (T*)G->step, ctrl, s));
  } else {
    if (G->nrows > 0) CKL(launch_proj_U_rows<T>(G->g, rows_dev(G), G->u64, G->uhi, G->ulo, (T*)G->step, ctrl, s));
    if (G->contact) CKL(launch_contact_proj_U<T>(ca, G->u64, G->uhi, G->ulo, (T*)G->step, s));
    CKL(launch_ctrl_end(ctrl, s));
  }
  prof_mark(8, s);
  return DTT_OK;
}

dtt_status enqueue_iter_any(dtt_grid* G, int acv_on, bool acv) {
  return G->prec == DTT_PREC_FP64 ? enqueue_iteration<double>(G, acv_on, acv)
                                  : enqueue_iteration<float>(G, acv_on, acv);
}

// The whole solve as one CUDA graph: a conditional WHILE node whose body is one round
// (`round` enqueues it on stream s, which may fork to other streams and join back) followed
// by the loop condition (k_loop_continue: another round while a grid runs, at most
// rounds[1] rounds; rounds[0] counts them).  *looped = false, with no graph, when the
// driver does not take conditional nodes (or DTT_GRAPH_LOOP=0 asks for the host loop); the
// caller then captures one round and loops on the host.
template <typename F>
dtt_status build_loop_graph(cudaStream_t s, F&& round, Ctrl* const* ctrls, const Ctrl* one, int n, int* rounds,
                            cudaGraphExec_t* exec, bool* looped) {
  *looped = false;
  *exec = nullptr;
  if (const char* v = std::getenv("DTT_GRAPH_LOOP"))
    if (v[0] == '0') return DTT_OK;
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h{};
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return DTT_OK;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return DTT_OK;
  }
  dtt_status st = round();
  if (st == DTT_OK && launch_loop_continue(ctrls, one, n, h, rounds, 0, s) != 0)
    st = fail(DTT_ERR_CUDA, "loop condition launch");
  cudaGraph_t got = nullptr;
  e = cudaStreamEndCapture(s, &got);
  if (st != DTT_OK || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    if (st != DTT_OK) return st;
    return fail(DTT_ERR_CUDA, std::string("loop capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return fail(DTT_ERR_CUDA, std::string("cudaGraphInstantiate (loop): ") + cudaGetErrorString(e));
  }
  *looped = true;
  return DTT_OK;
}

// Resets the loop's round counter and sets its cap (before each launch of a loop graph).
dtt_status arm_loop(int* rounds, int max_rounds, cudaStream_t s) {
  const int v[2] = {0, max_rounds};
  CK(cudaMemcpyAsync(rounds, v, sizeof(v), cudaMemcpyHostToDevice, s));
  return DTT_OK;
}

dtt_status build_graph(dtt_grid* G, int acv_on, bool acv, int iters) {
  invalidate_graph(G);
  if (!G->d_rounds) {
    dtt_status st = dalloc(&G->d_rounds, 2 * sizeof(int));
    if (st != DTT_OK) return st;
  }
  auto round = [&]() {
    dtt_status st = DTT_OK;
    for (int k = 0; k < iters && st == DTT_OK; ++k) st = enqueue_iter_any(G, acv_on, acv);
    return st;
  };
  bool looped = false;
  dtt_status st = build_loop_graph(G->stream, round, nullptr, G->d_ctrl, 1, G->d_rounds, &G->gexec, &looped);
  if (st != DTT_OK) return st;
  G->g_loop = looped;
  if (!looped) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeThreadLocal));
    st = round();
    cudaError_t e = cudaStreamEndCapture(G->stream, &graph);
    if (st != DTT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(DTT_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&G->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      G->gexec = nullptr;
      return fail(DTT_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
  }
  G->g_key = acv_on * 1000000 + (acv ? 100000 : 0) + iters;
  return DTT_OK;
}

dtt_status to_grid_u(dtt_grid* G, const double* u, int is_dev) {
  // copy a float64 field into the grid's u~ storage
  const size_t n3 = (size_t)(3 * G->NN);
  const double* src = u;
  if (!is_dev) {
    CK(cudaMemcpyAsync(G->op_d, u, n3 * sizeof(double), cudaMemcpyHostToDevice, G->stream));
    src = G->op_d;
  }
  if (G->prec == DTT_PREC_FP64) {
    if (src != G->u64) CK(cudaMemcpyAsync(G->u64, src, n3 * sizeof(double), cudaMemcpyDeviceToDevice, G->stream));
  } else {
    CKL(launch_split((long long)n3, src, G->uhi, G->ulo, G->stream));
  }
  return DTT_OK;
}

dtt_status zero_dirichlet(dtt_grid* G) {
  // enforce u~ = 0 on Dirichlet-face DOFs
  CKL(launch_zero_dirichlet(G->g, G->u64, G->uhi, G->ulo, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  return DTT_OK;
}

dtt_status ensure_ops(dtt_grid* G) {
  if (G->op_t1) return DTT_OK;
  size_t n3 = (size_t)(3 * G->NN);
  dtt_status s = dalloc(&G->op_t1, n3 * G->esz);
  if (s == DTT_OK) s = dalloc(&G->op_t2, n3 * G->esz);
  return s;
}

void free_rows(dtt_grid* G) {
  dfree(G->d_ptr);
  dfree(G->d_dof);
  dfree(G->d_a);
  dfree(G->d_b);
  dfree(G->d_target);
  dfree(G->d_mult);
  dfree(G->d_ab);
  dfree(G->d_aa);
}

void free_contact(dtt_grid* G) {
  dfree(G->d_face);
  dfree(G->d_active);
  dfree(G->d_vgap);
  dfree(G->d_vreact);
  dfree(G->d_vgap_prev);
  dfree(G->d_vreact_prev);
  dfree(G->d_gap);
  dfree(G->d_fn);
  dfree(G->d_nvec);
  dfree(G->d_active_saved);
  G->nface = 0;
  G->contact = false;
  G->contact_given = false;
}

}  // namespace

extern "C" {

const char* dtt_last_error(void) { return g_err.c_str(); }
const char* dtt_version(void) { return "libdtt 0.1 (sm_103a)"; }

dtt_status dtt_grid_create(dtt_grid** out, const int32_t nvox[3], double h, const int32_t bc[18], int32_t scheme,
                           int32_t precision, void* stream) {
  if (!out || !nvox || !bc) return fail(DTT_ERR_ARG, "null argument");
  *out = nullptr;
  if (!(h > 0.0)) return fail(DTT_ERR_ARG, "h must be > 0");
  if (scheme != DTT_SCHEME_TETRA2 && scheme != DTT_SCHEME_HEX1) return fail(DTT_ERR_ARG, "unknown scheme");
  if (precision != DTT_PREC_FP64 && precision != DTT_PREC_MIXED) return fail(DTT_ERR_ARG, "unknown precision");
  for (int d = 0; d < 3; ++d)
    if (nvox[d] < 2 || nvox[d] > 4096) return fail(DTT_ERR_ARG, "nvox must be in [2, 4096]");
  for (int q = 0; q < 18; ++q)
    if (bc[q] < 0 || bc[q] > 2) return fail(DTT_ERR_ARG, "bc code must be 0, 1 or 2");
  dtt_grid* G = new dtt_grid();
  static std::atomic<unsigned long long> next_id{1};
  G->id = next_id.fetch_add(1);
  G->prec = precision;
  G->esz = precision == DTT_PREC_FP64 ? 8 : 4;
  G->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&G->device) != cudaSuccess) {
    delete G;
    return fail(DTT_ERR_CUDA, "cudaGetDevice failed");
  }
  G->g.h = h;
  G->g.scheme = scheme;
  for (int d = 0; d < 3; ++d) {
    G->g.nvox[d] = nvox[d];
    for (int f = 0; f < 2; ++f)
      for (int c = 0; c < 3; ++c) G->g.bc[d][f][c] = bc[d * 6 + f * 3 + c];
    int nper = 0;
    for (int c = 0; c < 3; ++c) {
      int t = ttype(G->g.bc[d][0][c], G->g.bc[d][1][c]);
      if (t < 0) { delete G; return fail(DTT_ERR_BC, "periodic must be set on both faces of an axis"); }
      G->types[c][d] = t;
      nper += (t == T_DHT);
    }
    if (nper != 0 && nper != 3) { delete G; return fail(DTT_ERR_BC, "an axis is periodic for all components or none"); }
    G->g.periodic[d] = nper == 3;
    G->g.nn[d] = G->g.periodic[d] ? nvox[d] : nvox[d] + 1;
  }
  if (!G->stream) {
    if (cudaStreamCreate(&G->stream) != cudaSuccess) {
      delete G;
      return fail(DTT_ERR_CUDA, "cudaStreamCreate failed");
    }
    G->own_stream = true;
  }
  G->NN = (long long)G->g.nn[0] * G->g.nn[1] * G->g.nn[2];
  G->NV = (long long)nvox[0] * nvox[1] * nvox[2];
  G->g.nnodes = G->NN;
  for (int c = 0; c < 3; ++c) G->has_null[c] = comp_has_null(G, c);

  const size_t n3 = (size_t)(3 * G->NN);
  dtt_status s = DTT_OK;
  if (precision == DTT_PREC_FP64) s = dalloc(&G->u64, n3 * sizeof(double));
  else {
    s = dalloc(&G->uhi, n3 * sizeof(float));
    if (s == DTT_OK) s = dalloc(&G->ulo, n3 * sizeof(float));
  }
  for (int k = 0; k < 5 && s == DTT_OK; ++k) s = dalloc(&G->S[k], n3 * G->esz);
  for (int k = 0; k < 4 && s == DTT_OK; ++k) s = dalloc(&G->R[k], n3 * G->esz);
  for (int k = 0; k < 4 && s == DTT_OK; ++k) s = dalloc(&G->Gr[k], n3 * G->esz);
  if (s == DTT_OK) G->gbuf = G->Gr[0];
  if (s == DTT_OK) s = dalloc(&G->step, n3 * G->esz);
  if (s == DTT_OK) s = dalloc(&G->spec, n3 * G->esz);
  if (s == DTT_OK) s = dalloc(&G->spec2, n3 * G->esz);
  if (s == DTT_OK) s = dalloc(&G->d_Sring, 5 * sizeof(void*));
  if (s == DTT_OK) s = dalloc(&G->d_Rring, 4 * sizeof(void*));
  if (s == DTT_OK) s = dalloc(&G->d_Gring, 4 * sizeof(void*));
  if (s == DTT_OK) s = dalloc(&G->d_Gown, 4 * sizeof(void*));
  if (s == DTT_OK) s = dalloc(&G->phase, (size_t)G->NV);
  if (s == DTT_OK) s = dalloc(&G->d_lam, MAX_PHASE * sizeof(double));
  if (s == DTT_OK) s = dalloc(&G->d_mu, MAX_PHASE * sizeof(double));
  if (s == DTT_OK) s = dalloc(&G->cmask, (size_t)G->NN);
  if (s == DTT_OK) s = dalloc(&G->d_ctrl, sizeof(Ctrl));
  if (s == DTT_OK) s = dalloc(&G->op_d, n3 * sizeof(double));
  if (s == DTT_OK) {
    cudaError_t e = cudaMallocHost((void**)&G->h_ctrl, sizeof(Ctrl));
    if (e != cudaSuccess) s = fail(DTT_ERR_OOM, "cudaMallocHost");
  }
  if (s == DTT_OK) s = ensure_partials(G);
  if (s != DTT_OK) { dtt_grid_destroy(G); return s; }
  // transform tables
  for (int c = 0; c < 3 && s == DTT_OK; ++c)
    for (int d = 0; d < 3 && s == DTT_OK; ++d) {
      std::vector<double> F, B, cq, cc;
      int nn = G->g.nn[d];
      build_axis(G->types[c][d], nvox[d], nn, F, B, cq, cc);
      s = dalloc(&G->fwd[c][d], (size_t)nn * nn * G->esz);
      if (s == DTT_OK) s = dalloc(&G->inv[c][d], (size_t)nn * nn * G->esz);
      if (s == DTT_OK) s = dalloc(&G->sin2q[c][d], (size_t)nn * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->cos2q[c][d], (size_t)nn * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->sin2q_f[c][d], (size_t)nn * sizeof(float));
      if (s == DTT_OK) s = dalloc(&G->cos2q_f[c][d], (size_t)nn * sizeof(float));
      if (s != DTT_OK) break;
      if (G->esz == 8) {
        cudaMemcpy(G->fwd[c][d], F.data(), F.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(G->inv[c][d], B.data(), B.size() * 8, cudaMemcpyHostToDevice);
      } else {
        std::vector<float> Ff(F.begin(), F.end()), Bf(B.begin(), B.end());
        cudaMemcpy(G->fwd[c][d], Ff.data(), Ff.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(G->inv[c][d], Bf.data(), Bf.size() * 4, cudaMemcpyHostToDevice);
      }
      cudaMemcpy(G->sin2q[c][d], cq.data(), cq.size() * 8, cudaMemcpyHostToDevice);
      cudaMemcpy(G->cos2q[c][d], cc.data(), cc.size() * 8, cudaMemcpyHostToDevice);
      {
        std::vector<float> cqf(cq.begin(), cq.end()), ccf(cc.begin(), cc.end());
        cudaMemcpy(G->sin2q_f[c][d], cqf.data(), cqf.size() * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(G->cos2q_f[c][d], ccf.data(), ccf.size() * 4, cudaMemcpyHostToDevice);
      }
    }
  for (int d = 0; d < 3 && s == DTT_OK; ++d) s = build_fft_axis(G, d);
  // DTT_WFFT=0 keeps the Stockham passes, DTT_EXACT_R=0 the residual's A0 Delta form
  // (route comparisons; read once, at creation)
  if (const char* e = std::getenv("DTT_WFFT")) G->fft_warp = (e[0] == '0') ? 0 : 1;
  if (const char* e = std::getenv("DTT_EXACT_R")) G->exact_ok = (e[0] == '0') ? 0 : 1;
  if (s == DTT_OK && precision == DTT_PREC_MIXED) s = build_tz(G);
  if (s == DTT_OK) {
    cudaError_t e = cudaMemcpy(G->d_Sring, G->S, 5 * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G->d_Rring, G->R, 4 * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G->d_Gring, G->Gr, 4 * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G->d_Gown, G->Gr, 4 * sizeof(void*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(G->cmask, 0, (size_t)G->NN);
    if (e == cudaSuccess && s == DTT_OK) s = build_tile_z(G, std::vector<long long>());
    if (e == cudaSuccess) e = G->u64 ? cudaMemset(G->u64, 0, n3 * 8) : cudaMemset(G->uhi, 0, n3 * 4);
    if (e == cudaSuccess && G->ulo) e = cudaMemset(G->ulo, 0, n3 * 4);
    if (e != cudaSuccess) s = fail(DTT_ERR_CUDA, std::string("set-up copy: ") + cudaGetErrorString(e));
  }
  if (s != DTT_OK) { dtt_grid_destroy(G); return s; }
  *out = G;
  return DTT_OK;
}

void dtt_grid_destroy(dtt_grid* G) {
  if (!G) return;
  if (G->stream) cudaStreamSynchronize(G->stream);
  else cudaDeviceSynchronize();
  invalidate_graph(G);
  dfree(G->u64);
  dfree(G->uhi);
  dfree(G->ulo);
  dfree(G->tz_err);
  for (auto& p : G->S) dfree(p);
  for (auto& p : G->R) dfree(p);
  for (auto& p : G->Gr) dfree(p);
  G->gbuf = nullptr;
  dfree(G->step);
  dfree(G->spec);
  dfree(G->spec2);
  dfree(G->d_Sring);
  dfree(G->d_Rring);
  dfree(G->d_Gring);
  dfree(G->d_Gown);
  dfree(G->phase);
  dfree(G->d_lam);
  dfree(G->d_mu);
  dfree(G->cmask);
  dfree(G->d_ctrl);
  dfree(G->d_part);
  dfree(G->op_d);
  dfree(G->op_t1);
  dfree(G->op_t2);
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      dfree(G->fwd[c][d]);
      dfree(G->inv[c][d]);
      dfree(G->sin2q[c][d]);
      dfree(G->cos2q[c][d]);
      dfree(G->sin2q_f[c][d]);
      dfree(G->cos2q_f[c][d]);
      if (d == 0) dfree(G->tz_mat[c]);
      if (c == 0) {
        dfree(G->iso_s[d]);
        dfree(G->iso_c[d]);
        dfree(G->iso_sf[d]);
        dfree(G->iso_cf[d]);
        dfree(G->iso_valid[d]);
      }
    }
  for (int d = 0; d < 3; ++d) {
    dfree(G->fft_tw[d]);
    dfree(G->fft_ph[d]);
    dfree(G->fft_tw1[d]);
  }
  {
    dfree(G->d_tile_z);
    dfree(G->d_rounds);
  }
  free_rows(G);
  free_contact(G);
  if (G->h_ctrl) cudaFreeHost(G->h_ctrl);
  if (G->own_stream) cudaStreamDestroy(G->stream);
  delete G;
}

dtt_status dtt_grid_sizes(const dtt_grid* G, int64_t* n_nodes, int64_t* n_voxels, int32_t nn[3]) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (n_nodes) *n_nodes = G->NN;
  if (n_voxels) *n_voxels = G->NV;
  if (nn)
    for (int d = 0; d < 3; ++d) nn[d] = G->g.nn[d];
  return DTT_OK;
}

dtt_status dtt_set_material(dtt_grid* G, const uint8_t* phase, int32_t nphase, const double* lambda, const double* mu,
                            int32_t phase_is_device) {
  if (!G || !phase || !lambda || !mu) return fail(DTT_ERR_ARG, "null argument");
  if (nphase < 1 || nphase > MAX_PHASE) return fail(DTT_ERR_ARG, "nphase must be in [1, 256]");
  for (int q = 0; q < nphase; ++q)
    if (!(lambda[q] >= 0.0) || !(mu[q] >= 0.0) || !std::isfinite(lambda[q]) || !std::isfinite(mu[q]))
      return fail(DTT_ERR_ARG, "Lame coefficients must be finite and >= 0");
  if (!phase_is_device) {
    for (long long v = 0; v < G->NV; ++v)
      if (phase[v] >= nphase) return fail(DTT_ERR_ARG, "phase id >= nphase");
    CK(cudaMemcpy(G->phase, phase, (size_t)G->NV, cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(G->phase, phase, (size_t)G->NV, cudaMemcpyDeviceToDevice));
    std::vector<uint8_t> h((size_t)G->NV);
    CK(cudaMemcpy(h.data(), G->phase, (size_t)G->NV, cudaMemcpyDeviceToHost));
    for (uint8_t v : h)
      if (v >= nphase) return fail(DTT_ERR_ARG, "phase id >= nphase");
  }
  CK(cudaMemcpy(G->d_lam, lambda, nphase * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(G->d_mu, mu, nphase * sizeof(double), cudaMemcpyHostToDevice));
  // The captured iteration reads the phase ids and the Lame tables through device
  // pointers, with the phase count by value: new values for as many phases keep it valid.
  const bool same_layout = G->mat_set && G->nphase == nphase;
  G->nphase = nphase;
  G->mat_set = true;
  if (!same_layout) invalidate_graph(G);
  return DTT_OK;
}

dtt_status dtt_set_reference(dtt_grid* G, double lambda0, double mu0) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (!(mu0 > 0.0) || !(lambda0 >= 0.0) || !std::isfinite(lambda0) || !std::isfinite(mu0))
    return fail(DTT_ERR_ARG, "reference medium needs mu0 > 0, lambda0 >= 0");
  G->lam0 = lambda0;
  G->mu0 = mu0;
  G->ref_set = true;
  invalidate_graph(G);
  return DTT_OK;
}

// Normal mixed conditions on every face (no periodic axis): the normal component's
// condition differs from both tangential components'.
// The isotropic medium's conditions (Section 3.2.3): every axis periodic for all
// components, or normal mixed on both of its faces.
static bool normal_mixed(const dtt_grid* G) {
  for (int d = 0; d < 3; ++d) {
    if (G->g.periodic[d]) {
      for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c)
          if (G->g.bc[d][f][c] != BC_P) return false;
      continue;
    }
    for (int f = 0; f < 2; ++f) {
      const int nrm = G->g.bc[d][f][d];
      for (int c = 0; c < 3; ++c)
        if (c != d && G->g.bc[d][f][c] == nrm) return false;
    }
  }
  return true;
}

// Per-axis tables of the isotropic medium: sin^2(q/2), cos^2(q/2) at each position from
// any component with a mode there (normal mixed conditions give the components the same
// q wherever they have a mode), and the bit set of those components.
static dtt_status build_iso_tables(dtt_grid* G) {
  for (int d = 0; d < 3; ++d) {
    const int nn = G->g.nn[d];
    std::vector<double> sq(nn, 0.0), cq(nn, 1.0);
    std::vector<uint8_t> valid(nn, 0);
    for (int c = 0; c < 3; ++c) {
      std::vector<double> F, B, cs, cc;
      build_axis(G->types[c][d], G->g.nvox[d], nn, F, B, cs, cc);
      for (int i = 0; i < nn; ++i) {
        // a position carries a mode when the forward transform's row is not all zero
        bool any = false;
        for (int j = 0; j < nn && !any; ++j) any = F[(size_t)i * nn + j] != 0.0;
        if (!any) continue;
        valid[i] |= (uint8_t)(1 << c);
        sq[i] = cs[i];
        cq[i] = cc[i];
      }
    }
    std::vector<float> sqf(sq.begin(), sq.end()), cqf(cq.begin(), cq.end());
    dtt_status st = DTT_OK;
    if (!G->iso_s[d]) {
      st = dalloc(&G->iso_s[d], nn * sizeof(double));
      if (st == DTT_OK) st = dalloc(&G->iso_c[d], nn * sizeof(double));
      if (st == DTT_OK) st = dalloc(&G->iso_sf[d], nn * sizeof(float));
      if (st == DTT_OK) st = dalloc(&G->iso_cf[d], nn * sizeof(float));
      if (st == DTT_OK) st = dalloc(&G->iso_valid[d], nn);
      if (st != DTT_OK) return st;
    }
    CK(cudaMemcpy(G->iso_s[d], sq.data(), nn * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->iso_c[d], cq.data(), nn * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->iso_sf[d], sqf.data(), nn * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->iso_cf[d], cqf.data(), nn * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->iso_valid[d], valid.data(), nn, cudaMemcpyHostToDevice));
  }
  return DTT_OK;
}

dtt_status dtt_set_reference_medium(dtt_grid* G, int32_t medium) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (medium != DTT_MEDIUM_PAUX && medium != DTT_MEDIUM_ISOTROPIC)
    return fail(DTT_ERR_ARG, "medium must be DTT_MEDIUM_PAUX or DTT_MEDIUM_ISOTROPIC");
  const int iso = medium == DTT_MEDIUM_ISOTROPIC;
  if (iso && !normal_mixed(G))
    return fail(DTT_ERR_BC, "the isotropic reference medium needs, on every axis, periodic conditions for all "
                            "components or normal mixed conditions (normal component Dirichlet with tangential "
                            "Neumann, or the reverse) on both faces");
  if (iso && !G->iso_s[0]) {
    dtt_status st = build_iso_tables(G);
    if (st != DTT_OK) return st;
  }
  if (G->g.ref_iso != iso) {
    G->g.ref_iso = iso;
    invalidate_graph(G);
  }
  return DTT_OK;
}

dtt_status dtt_set_load(dtt_grid* G, const double eps_star[9]) {
  if (!G || !eps_star) return fail(DTT_ERR_ARG, "null argument");
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      double v = 0.5 * (eps_star[3 * p + q] + eps_star[3 * q + p]);
      if (!std::isfinite(v)) return fail(DTT_ERR_ARG, "eps* must be finite");
      G->eps[p][q] = v;
    }
  invalidate_graph(G);
  return DTT_OK;
}

dtt_status dtt_set_constraints(dtt_grid* G, int32_t n_rows, const int32_t* row_ptr, const int32_t* node,
                               const int8_t* comp, const double* a, const double* b, const double* value) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (n_rows < 0) return fail(DTT_ERR_ARG, "n_rows < 0");
  std::vector<int> ptr;
  std::vector<long long> dof;
  std::vector<double> va, vb, vv, vab, vaa;
  if (n_rows > 0) {
    if (!row_ptr || !node || !comp || !a || !value) return fail(DTT_ERR_ARG, "null constraint array");
    if (row_ptr[0] != 0) return fail(DTT_ERR_ARG, "row_ptr[0] must be 0");
    std::vector<uint8_t> seen((size_t)(3 * G->NN), 0);
    ptr.assign(row_ptr, row_ptr + n_rows + 1);
    for (int r = 0; r < n_rows; ++r) {
      if (row_ptr[r + 1] <= row_ptr[r]) return fail(DTT_ERR_ARG, "empty or decreasing row");
      double sab = 0.0, saa = 0.0;
      for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        if (node[e] < 0 || node[e] >= G->NN) return fail(DTT_ERR_ARG, "node index out of range");
        if (comp[e] < 0 || comp[e] > 2) return fail(DTT_ERR_ARG, "component must be 0, 1 or 2");
        if (!std::isfinite(a[e]) || (b && !std::isfinite(b[e]))) return fail(DTT_ERR_ARG, "non-finite weight");
        int c = comp[e];
        if (G->has_null[c])
          return fail(DTT_ERR_NULLMODE, "constraint on component " + std::to_string(c) +
                                             " whose Green symbol has null modes (give it a Dirichlet face)");
        bool dofok;
        double W;
        host_node_W(G, c, node[e], dofok, W);
        if (!dofok) return fail(DTT_ERR_ARG, "constraint entry on a Dirichlet-face DOF");
        long long d = (long long)c * G->NN + node[e];
        if (seen[(size_t)d]) return fail(DTT_ERR_OVERLAP, "constraint rows overlap");
        seen[(size_t)d] = 1;
        double bb = b ? b[e] : a[e];
        dof.push_back(d);
        va.push_back(a[e]);
        vb.push_back(bb);
        sab += a[e] * bb;
        saa += a[e] * a[e];
      }
      if (!(saa > 0.0) || sab == 0.0) return fail(DTT_ERR_ARG, "row with sum a^2 = 0 or sum a b = 0");
      if (!std::isfinite(value[r])) return fail(DTT_ERR_ARG, "non-finite constraint value");
      vv.push_back(value[r]);
      vab.push_back(sab);
      vaa.push_back(saa);
    }
  }
  // Rows of the same count and total length reuse the device buffers; the captured
  // iteration, which holds their addresses and the row count, then stays valid.
  const bool same_layout = n_rows == G->nrows && dof.size() == G->h_dof.size() && (n_rows == 0 || G->d_ptr);
  if (!same_layout) free_rows(G);
  G->nrows = n_rows;
  G->h_ptr = ptr;
  G->h_dof = dof;
  G->h_a = va;
  G->h_b = vb;
  G->h_val = vv;
  G->h_ab = vab;
  G->h_aa = vaa;
  if (n_rows > 0) {
    size_t ne = dof.size();
    dtt_status s = DTT_OK;
    if (!same_layout) {
      s = dalloc(&G->d_ptr, (n_rows + 1) * sizeof(int));
      if (s == DTT_OK) s = dalloc(&G->d_dof, ne * sizeof(long long));
      if (s == DTT_OK) s = dalloc(&G->d_a, ne * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->d_b, ne * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->d_target, n_rows * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->d_mult, n_rows * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->d_ab, n_rows * sizeof(double));
      if (s == DTT_OK) s = dalloc(&G->d_aa, n_rows * sizeof(double));
    }
    if (s != DTT_OK) { G->nrows = 0; invalidate_graph(G); return s; }
    CK(cudaMemcpy(G->d_ptr, ptr.data(), (n_rows + 1) * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->d_dof, dof.data(), ne * sizeof(long long), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->d_a, va.data(), ne * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->d_b, vb.data(), ne * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->d_ab, vab.data(), n_rows * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(G->d_aa, vaa.data(), n_rows * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(G->d_mult, 0, n_rows * sizeof(double)));
  }
  const double* part_before = G->d_part;
  dtt_status s = ensure_partials(G);
  if (s != DTT_OK) return s;
  if (!same_layout || G->d_part != part_before) invalidate_graph(G);
  return rebuild_cmask(G);
}

dtt_status dtt_set_indenter(dtt_grid* G, int32_t axis, int32_t face, const double center[3], double radius) {
  if (!G || !center) return fail(DTT_ERR_ARG, "null argument");
  if (axis < 0 || axis > 2 || face < 0 || face > 1) return fail(DTT_ERR_ARG, "axis in 0..2, face in 0..1");
  if (G->g.periodic[axis]) return fail(DTT_ERR_BC, "contact face on a periodic axis");
  if (!(radius > 0.0)) return fail(DTT_ERR_ARG, "radius must be > 0");
  for (int c = 0; c < 3; ++c)
    if (G->has_null[c]) return fail(DTT_ERR_NULLMODE, "contact needs components without Green null modes");
  free_contact(G);
  std::vector<long long> nodes;
  const int fi = face == 0 ? 0 : G->g.nn[axis] - 1;
  for (int k = 0; k < G->g.nn[2]; ++k)
    for (int j = 0; j < G->g.nn[1]; ++j)
      for (int i = 0; i < G->g.nn[0]; ++i) {
        int idx[3] = {i, j, k};
        if (idx[axis] != fi) continue;
        nodes.push_back(i + (long long)G->g.nn[0] * (j + (long long)G->g.nn[1] * k));
      }
  G->nface = (int)nodes.size();
  size_t nf = nodes.size();
  dtt_status s = dalloc(&G->d_face, nf * sizeof(long long));
  if (s == DTT_OK) s = dalloc(&G->d_active, nf);
  if (s == DTT_OK) s = dalloc(&G->d_vgap, nf);
  if (s == DTT_OK) s = dalloc(&G->d_vreact, nf);
  if (s == DTT_OK) s = dalloc(&G->d_vgap_prev, nf);
  if (s == DTT_OK) s = dalloc(&G->d_vreact_prev, nf);
  if (s == DTT_OK) s = dalloc(&G->d_gap, nf * sizeof(double));
  if (s == DTT_OK) s = dalloc(&G->d_fn, nf * sizeof(double));
  if (s == DTT_OK) s = dalloc(&G->d_nvec, 3 * nf * sizeof(double));
  if (s != DTT_OK) { free_contact(G); return s; }
  CK(cudaMemcpy(G->d_face, nodes.data(), nf * sizeof(long long), cudaMemcpyHostToDevice));
  CK(cudaMemset(G->d_active, 0, nf));
  CK(cudaMemset(G->d_fn, 0, nf * sizeof(double)));
  CK(cudaMemset(G->d_gap, 0, nf * sizeof(double)));
  CK(cudaMemset(G->d_nvec, 0, 3 * nf * sizeof(double)));
  G->contact = true;
  G->c_axis = axis;
  G->c_face = face;
  for (int c = 0; c < 3; ++c) G->center[c] = center[c];
  G->radius = radius;
  s = ensure_partials(G);
  if (s != DTT_OK) return s;
  invalidate_graph(G);
  return rebuild_cmask(G);
}

dtt_status dtt_move_indenter(dtt_grid* G, const double center[3]) {
  if (!G || !center) return fail(DTT_ERR_ARG, "null argument");
  if (!G->contact) return fail(DTT_ERR_STATE, "no indenter set");
  for (int c = 0; c < 3; ++c) {
    if (!std::isfinite(center[c])) return fail(DTT_ERR_ARG, "non-finite centre");
    G->center[c] = center[c];
  }
  invalidate_graph(G);
  return DTT_OK;
}

dtt_status dtt_clear_indenter(dtt_grid* G) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  free_contact(G);
  invalidate_graph(G);
  return rebuild_cmask(G);
}

}  // extern "C"

dtt_status dtt::set_guess_with_fallback(dtt_grid* G, const double* u_dev, const uint8_t* active_dev) {
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  if (G->prec == DTT_PREC_FP64) {
    CK(cudaMemcpyAsync(G->R[0], G->u64, n3 * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemcpyAsync(G->R[0], G->uhi, n3 * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(G->R[1], G->ulo, n3 * 4, cudaMemcpyDeviceToDevice, s));
  }
  dtt_status st = dtt_set_initial(G, u_dev, 1);
  if (st != DTT_OK) return st;
  if (active_dev && G->contact) {
    st = dtt_set_initial_contact(G, active_dev, 1);
    if (st != DTT_OK) return st;
  }
  G->fallback_saved = true;
  return DTT_OK;
}

extern "C" {

dtt_status dtt_set_initial_contact(dtt_grid* G, const uint8_t* active, int32_t ptr_is_device) {
  if (!G || !active) return fail(DTT_ERR_ARG, "null argument");
  if (!G->contact) return fail(DTT_ERR_STATE, "no indenter set");
  CK(cudaMemcpyAsync(G->d_active, active, (size_t)G->nface,
                     ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  G->contact_given = true;
  return DTT_OK;
}

dtt_status dtt_set_initial(dtt_grid* G, const double* u, int32_t ptr_is_device) {
  if (!G || !u) return fail(DTT_ERR_ARG, "null argument");
  dtt_status s = to_grid_u(G, u, ptr_is_device);
  if (s != DTT_OK) return s;
  CK(cudaStreamSynchronize(G->stream));
  return zero_dirichlet(G);
}

}  // extern "C"

namespace {

// Eq. 5 residual of the current u~ after the initial projections (rows, contact), as the
// first iteration of a solve would measure it (u~ is projected in place).
template <typename T>
dtt_status eval_start_residual(dtt_grid* G, double* r) {
  cudaStream_t s = G->stream;
  PartRegions pr = regions(G);
  Ctrl& c = *G->h_ctrl;
  std::memset(&c, 0, sizeof(Ctrl));
  c.max_iter = 1 << 30;
  c.acv_mod = 1;
  c.contact_on = G->contact ? 1 : 0;
  c.update_tol = 1e-2;
  c.no_stop = 1;
  Ctrl* ctrl = G->d_ctrl;
  CK(cudaMemcpyAsync(ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  ContactArgs ca = contact_args(G, pr.cont);
  if (G->contact) {
    CKL(launch_contact_init(ca, s, G->contact_given ? 1 : 0));
    CKL(launch_contact_proj_U<T>(ca, G->u64, G->uhi, G->ulo, nullptr, s));
  }
  if (G->nrows > 0) CKL(launch_proj_U_rows<T>(G->g, rows_dev(G), G->u64, G->uhi, G->ulo, nullptr, ctrl, s));
  ResidualArgs ra{};
  ra.g = G->g;
  ra.u64 = G->u64;
  ra.uhi = G->uhi;
  ra.ulo = G->ulo;
  ra.phase = G->phase;
  ra.lam = G->d_lam;
  ra.mu = G->d_mu;
  ra.nphase = G->nphase;
  ra.cmask = G->cmask;
  std::memcpy(ra.eps, G->eps, sizeof(ra.eps));
  ra.lam0 = G->lam0;
  ra.mu0 = G->mu0;
  ra.mode = 2;
  ra.pout = G->gbuf;
  ra.partials = pr.res;
  ra.ctrl = ctrl;
  CKL(launch_residual<T>(ra, s));
  if (G->nrows > 0)
    CKL(launch_proj_P_rows<T>(G->g, rows_dev(G), (T*)G->gbuf, G->d_Sring, G->d_Rring, 0, 0, pr.proj, ctrl, s));
  if (G->contact) CKL(launch_contact_eval<T>(ca, (T*)G->gbuf, G->d_Sring, G->d_Rring, 0, 0, s));
  CKL(launch_ctrl_residual(ctrl, pr.res, pr.nres, pr.proj, G->nrows > 0 ? pr.nproj : 0, pr.cont, pr.ncont, G->g.h,
                           G->NN, G->NV, s));
  CK(cudaMemcpyAsync(G->h_ctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *r = G->h_ctrl->r;
  return DTT_OK;
}

// DTT_INIT_GUESS: keep the supplied u~ only if its starting residual is below the plain
// start's: u~ = 0, or the previous increment's u~ when the guess was set over it
// (set_guess_with_fallback).  A contact zone set with the guess is the guess's; the plain
// start takes the zone {g < 0} of its own field.
dtt_status choose_start(dtt_grid* G) {
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  const bool f64 = G->prec == DTT_PREC_FP64;
  const bool zone = G->contact && G->contact_given;
  double rg = 0.0, r0 = 0.0;
  dtt_status st = f64 ? eval_start_residual<double>(G, &rg) : eval_start_residual<float>(G, &rg);
  if (st != DTT_OK) return st;
  if (zone) {
    if (!G->d_active_saved && (st = dalloc(&G->d_active_saved, (size_t)G->nface)) != DTT_OK) return st;
    CK(cudaMemcpyAsync(G->d_active_saved, G->d_active, (size_t)G->nface, cudaMemcpyDeviceToDevice, s));
  }
  // the guess to S[3] / S[4]; the plain start into u~
  if (f64) {
    CK(cudaMemcpyAsync(G->S[4], G->u64, n3 * 8, cudaMemcpyDeviceToDevice, s));
    if (G->fallback_saved) CK(cudaMemcpyAsync(G->u64, G->R[0], n3 * 8, cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemsetAsync(G->u64, 0, n3 * 8, s));
  } else {
    CK(cudaMemcpyAsync(G->S[3], G->uhi, n3 * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(G->S[4], G->ulo, n3 * 4, cudaMemcpyDeviceToDevice, s));
    if (G->fallback_saved) {
      CK(cudaMemcpyAsync(G->uhi, G->R[0], n3 * 4, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(G->ulo, G->R[1], n3 * 4, cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemsetAsync(G->uhi, 0, n3 * 4, s));
      CK(cudaMemsetAsync(G->ulo, 0, n3 * 4, s));
    }
  }
  const bool had_fallback = G->fallback_saved;
  G->contact_given = false;
  G->fallback_saved = false;
  st = f64 ? eval_start_residual<double>(G, &r0) : eval_start_residual<float>(G, &r0);
  if (st != DTT_OK) return st;
  G->start_guess = (std::isfinite(rg) && rg < r0) ? 1 : 0;
  G->start_r = G->start_guess ? rg : r0;
  if (!G->start_guess) {
    // the plain start as it was before its evaluation projected it: the solve's own start
    // then matches a plain solve exactly
    if (f64) {
      if (had_fallback) CK(cudaMemcpyAsync(G->u64, G->R[0], n3 * 8, cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemsetAsync(G->u64, 0, n3 * 8, s));
    } else if (had_fallback) {
      CK(cudaMemcpyAsync(G->uhi, G->R[0], n3 * 4, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(G->ulo, G->R[1], n3 * 4, cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemsetAsync(G->uhi, 0, n3 * 4, s));
      CK(cudaMemsetAsync(G->ulo, 0, n3 * 4, s));
    }
  }
  if (G->start_guess) {
    if (f64) {
      CK(cudaMemcpyAsync(G->u64, G->S[4], n3 * 8, cudaMemcpyDeviceToDevice, s));
    } else {
      CK(cudaMemcpyAsync(G->uhi, G->S[3], n3 * 4, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(G->ulo, G->S[4], n3 * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (zone) {
      CK(cudaMemcpyAsync(G->d_active, G->d_active_saved, (size_t)G->nface, cudaMemcpyDeviceToDevice, s));
      G->contact_given = true;
    }
  }
  CK(cudaStreamSynchronize(s));
  return DTT_OK;
}

dtt_status check_solve(const dtt_grid* G, const dtt_solve_opts* opts) {
  if (!G || !opts) return fail(DTT_ERR_ARG, "null argument");
  if (!G->mat_set) return fail(DTT_ERR_STATE, "dtt_set_material not called");
  if (!G->ref_set) return fail(DTT_ERR_STATE, "dtt_set_reference not called");
  if (!(opts->tol >= 0.0) || opts->max_iter < 0) return fail(DTT_ERR_ARG, "tol >= 0 and max_iter >= 0 required");
  if (opts->acv_mod < 0) return fail(DTT_ERR_ARG, "acv_mod >= 0");
  if (opts->acv_on != DTT_ACV_U && opts->acv_on != DTT_ACV_P) return fail(DTT_ERR_ARG, "acv_on must be 0 or 1");
  if (opts->acv_on == DTT_ACV_U && G->prec != DTT_PREC_FP64 && opts->acv_mod > 0)
    return fail(DTT_ERR_ARG, "ACV on u~ is available in the FP64 path only");
  if (opts->init != DTT_INIT_ZERO && opts->init != DTT_INIT_PREVIOUS && opts->init != DTT_INIT_GUESS)
    return fail(DTT_ERR_ARG, "init must be 0, 1 or 2");
  return DTT_OK;
}

// Everything a solve does before its first iteration: initial u~, row targets, a fresh
// control block, zeroed rings, initial projections (all on the grid's stream).
dtt_status prepare_solve(dtt_grid* G, const dtt_solve_opts* opts) {
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  if (opts->init == DTT_INIT_ZERO) {
    if (G->u64) CK(cudaMemsetAsync(G->u64, 0, n3 * 8, s));
    else {
      CK(cudaMemsetAsync(G->uhi, 0, n3 * 4, s));
      CK(cudaMemsetAsync(G->ulo, 0, n3 * 4, s));
    }
  }
  // targets on u~ (U - A u*)
  if (G->nrows > 0) {
    std::vector<double> tg(G->nrows);
    for (int r = 0; r < G->nrows; ++r) {
      double su = 0.0;
      for (int e = G->h_ptr[r]; e < G->h_ptr[r + 1]; ++e) {
        long long d = G->h_dof[e];
        int c = (int)(d / G->NN);
        su += G->h_a[e] * host_ustar(G, c, d - c * G->NN);
      }
      tg[r] = G->h_val[r] - su;
    }
    CK(cudaMemcpyAsync(G->d_target, tg.data(), G->nrows * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  G->start_guess = 0;
  G->start_r = 0.0;
  if (opts->init == DTT_INIT_GUESS) {
    dtt_status st = choose_start(G);
    if (st != DTT_OK) return st;
  }
  // control block
  Ctrl& c = *G->h_ctrl;
  std::memset(&c, 0, sizeof(Ctrl));
  c.max_iter = opts->max_iter;
  c.acv_mod = opts->acv_mod > 0 ? opts->acv_mod : 1;
  c.acv_on = opts->acv_on;
  c.contact_on = G->contact ? 1 : 0;
  c.tol = opts->tol;
  c.update_tol = opts->update_tol > 0.0 ? opts->update_tol : 1e-2;
  c.acv_pivot = opts->acv_pivot > 0.0 ? opts->acv_pivot : 1e-14;
  CK(cudaMemcpyAsync(G->d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  for (int k = 0; k < 5; ++k) CK(cudaMemsetAsync(G->S[k], 0, n3 * G->esz, s));
  for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(G->R[k], 0, n3 * G->esz, s));
  for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(G->Gr[k], 0, n3 * G->esz, s));
  // the Green-input ring points at the own buffers again (a solve may leave aliases of p)
  CK(cudaMemcpyAsync(G->d_Gring, G->d_Gown, 4 * sizeof(void*), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(G->step, 0, n3 * G->esz, s));
  PartRegions pr = regions(G);
  ContactArgs ca = contact_args(G, pr.cont);
  if (G->contact) {
    CKL(launch_contact_init(ca, s, G->contact_given ? 1 : 0));
    G->contact_given = false;   // one start only
    if (G->prec == DTT_PREC_FP64) CKL(launch_contact_proj_U<double>(ca, G->u64, G->uhi, G->ulo, nullptr, s));
    else CKL(launch_contact_proj_U<float>(ca, G->u64, G->uhi, G->ulo, nullptr, s));
  }
  if (G->nrows > 0) {
    if (G->prec == DTT_PREC_FP64)
      CKL(launch_proj_U_rows<double>(G->g, rows_dev(G), G->u64, G->uhi, G->ulo, nullptr, G->d_ctrl, s));
    else
      CKL(launch_proj_U_rows<float>(G->g, rows_dev(G), G->u64, G->uhi, G->ulo, nullptr, G->d_ctrl, s));
  }
  return DTT_OK;
}

// Reads the final control block and fills the report (after the grid's work has finished).
dtt_status finish_solve(dtt_grid* G, std::chrono::steady_clock::time_point t0, dtt_report* rep) {
  cudaStream_t s = G->stream;
  CK(cudaMemcpyAsync(G->h_ctrl, G->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (G->tz_ok) {
    dtt_status te = check_tz(G);
    if (te != DTT_OK) return te;
  }
  G->last = *G->h_ctrl;
  G->solved = true;
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  dtt_status st = DTT_OK;
  if (G->last.done == 2 || G->last.done == 0) st = DTT_ERR_NOT_CONVERGED;
  if (G->last.done == 3) st = DTT_ERR_DIVERGED;
  if (rep) {
    rep->iterations = G->last.iter;
    rep->accelerations = G->last.n_accel;
    rep->active_set_updates = G->last.n_updates;
    rep->status = st;
    rep->residual = G->last.r;
    rep->seconds = secs;
    rep->start_from_guess = G->start_guess;
    rep->start_residual = G->start_r;
  }
  if (st == DTT_ERR_NOT_CONVERGED) g_err = "iteration cap reached";
  if (st == DTT_ERR_DIVERGED) g_err = "residual diverged";
  return st;
}

int graph_iters_of(const dtt_solve_opts* opts) { return opts->graph_iters > 0 ? opts->graph_iters : 8; }
int graph_key_of(const dtt_solve_opts* opts) {
  return opts->acv_on * 1000000 + (opts->acv_mod > 0 ? 100000 : 0) + graph_iters_of(opts);
}

}  // namespace

extern "C" {

dtt_status dtt_solve_step(dtt_grid* G, const dtt_solve_opts* opts, dtt_report* rep) {
  dtt_status st0 = check_solve(G, opts);
  if (st0 != DTT_OK) return st0;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = G->stream;
  st0 = prepare_solve(G, opts);
  if (st0 != DTT_OK) return st0;
  const bool acv = opts->acv_mod > 0;
  const int iters = graph_iters_of(opts);
  const int key = graph_key_of(opts);
  if (!G->gexec || G->g_key != key) {
    dtt_status st = build_graph(G, opts->acv_on, acv, iters);
    if (st != DTT_OK) return st;
  }
  long long launched = 0;
  const long long cap = (long long)opts->max_iter + 2LL * iters + 8;
  if (G->g_loop) {
    // one launch runs the solve to its end (the device loop stops at max_iter; the round
    // cap only guards it)
    dtt_status st = arm_loop(G->d_rounds, (int)std::min<long long>(cap / iters + 2, 1 << 30), s);
    if (st != DTT_OK) return st;
    CK(cudaGraphLaunch(G->gexec, s));
    return finish_solve(G, t0, rep);
  }
  while (true) {
    CK(cudaGraphLaunch(G->gexec, s));
    launched += iters;
    CK(cudaMemcpyAsync(G->h_ctrl, G->d_ctrl, 64, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (G->h_ctrl->done) break;
    if (launched > cap) break;   // cannot happen: the device stops at max_iter
  }
  return finish_solve(G, t0, rep);
}

dtt_status dtt_get_history(const dtt_grid* G, double* hist, int32_t* n) {
  if (!G || !n) return fail(DTT_ERR_ARG, "null argument");
  int m = std::min(G->last.hist_len, *n);
  if (hist)
    for (int k = 0; k < m; ++k) hist[k] = G->last.hist[k];
  *n = G->last.hist_len;
  return DTT_OK;
}

// Stress at the integration points into `out` (n_voxels x n_ip x ncomp), ncomp 6 or 9.
static dtt_status stress_to(dtt_grid* G, const double* src, double* out, int full, int32_t ptr_is_device) {
  cudaStream_t s = G->stream;
  if (!G->mat_set) return fail(DTT_ERR_STATE, "material not set");
  size_t ns = (size_t)G->NV * kIP[G->g.scheme] * (full ? 9 : 6);
  double* buf = nullptr;
  dtt_status st = dalloc(&buf, ns * sizeof(double));
  if (st != DTT_OK) return st;
  int rc = launch_stress_out(G->g, src, G->phase, G->d_lam, G->d_mu, G->eps, full, buf, s);
  if (rc) { dfree(buf); return fail(DTT_ERR_CUDA, "stress kernel launch"); }
  cudaError_t e = cudaMemcpyAsync(out, buf, ns * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  dfree(buf);
  if (e != cudaSuccess) return fail(DTT_ERR_CUDA, cudaGetErrorString(e));
  return DTT_OK;
}

// u~ as float64 on the device (the mixed path joins its float-float pair into op_d).
static dtt_status u_f64(dtt_grid* G, const double** src) {
  *src = G->u64;
  if (!*src) {
    CKL(launch_join((long long)(3 * G->NN), G->uhi, G->ulo, G->op_d, G->stream));
    *src = G->op_d;
  }
  return DTT_OK;
}

dtt_status dtt_get_fields(dtt_grid* G, double* u, double* sigma, int32_t ptr_is_device) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  const size_t n3 = (size_t)(3 * G->NN);
  cudaStream_t s = G->stream;
  const double* src = nullptr;
  dtt_status st = u_f64(G, &src);
  if (st != DTT_OK) return st;
  if (u) CK(cudaMemcpyAsync(u, src, n3 * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (sigma) {
    st = stress_to(G, src, sigma, 0, ptr_is_device);
    if (st != DTT_OK) return st;
  }
  CK(cudaStreamSynchronize(s));
  return DTT_OK;
}

dtt_status dtt_get_stress_tensor(dtt_grid* G, double* tensor, int32_t ptr_is_device) {
  if (!G || !tensor) return fail(DTT_ERR_ARG, "null argument");
  const double* src = nullptr;
  dtt_status st = u_f64(G, &src);
  if (st != DTT_OK) return st;
  st = stress_to(G, src, tensor, 1, ptr_is_device);
  if (st != DTT_OK) return st;
  CK(cudaStreamSynchronize(G->stream));
  return DTT_OK;
}

dtt_status dtt_get_min_jacobian(dtt_grid* G, double* det_min) {
  if (!G || !det_min) return fail(DTT_ERR_ARG, "null argument");
  const double* src = nullptr;
  dtt_status st = u_f64(G, &src);
  if (st != DTT_OK) return st;
  const int nb = min_jacobian_blocks(G->g);
  double* buf = nullptr;
  st = dalloc(&buf, (size_t)nb * sizeof(double));
  if (st != DTT_OK) return st;
  std::vector<double> h(nb);
  int rc = launch_min_jacobian(G->g, src, G->eps, buf, G->stream);
  cudaError_t e = rc ? (cudaError_t)rc
                     : cudaMemcpyAsync(h.data(), buf, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, G->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
  dfree(buf);
  if (e != cudaSuccess) return fail(DTT_ERR_CUDA, cudaGetErrorString(e));
  double m = h[0];
  for (int b = 1; b < nb; ++b) m = std::min(m, h[b]);
  *det_min = m;
  return DTT_OK;
}

dtt_status dtt_set_kinematics(dtt_grid* G, int32_t kinematics) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (kinematics != DTT_SMALL_STRAIN && kinematics != DTT_FINITE_STRAIN)
    return fail(DTT_ERR_ARG, "kinematics must be DTT_SMALL_STRAIN or DTT_FINITE_STRAIN");
  const int fs = kinematics == DTT_FINITE_STRAIN;
  if (G->g.finite_strain != fs) {
    G->g.finite_strain = fs;
    invalidate_graph(G);
  }
  return DTT_OK;
}

dtt_status dtt_get_reactions(dtt_grid* G, double* per_row, double total[3]) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  std::vector<double> f(G->nrows);
  if (G->nrows > 0) CK(cudaMemcpy(f.data(), G->d_mult, G->nrows * sizeof(double), cudaMemcpyDeviceToHost));
  double tot[3] = {0, 0, 0};
  const double h3 = G->g.h * G->g.h * G->g.h;
  for (int r = 0; r < G->nrows; ++r) {
    double pr = 0.0;
    for (int e = G->h_ptr[r]; e < G->h_ptr[r + 1]; ++e) {
      long long d = G->h_dof[e];
      int c = (int)(d / G->NN);
      bool dof;
      double W;
      host_node_W(G, c, d - c * G->NN, dof, W);
      double v = h3 * W * G->h_b[e] * f[r];
      pr += v;
      tot[c] += v;
    }
    if (per_row) per_row[r] = pr;
  }
  if (total)
    for (int c = 0; c < 3; ++c) total[c] = tot[c];
  return DTT_OK;
}

dtt_status dtt_get_contact(dtt_grid* G, int32_t* n_face, uint8_t* active, double* gap, double* fn, double force[3]) {
  if (!G) return fail(DTT_ERR_ARG, "null grid");
  if (n_face) *n_face = G->nface;
  if (!G->contact) {
    if (force) force[0] = force[1] = force[2] = 0.0;
    return DTT_OK;
  }
  size_t nf = G->nface;
  std::vector<uint8_t> act(nf);
  std::vector<double> f(nf), nv(3 * nf);
  CK(cudaMemcpy(act.data(), G->d_active, nf, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(f.data(), G->d_fn, nf * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(nv.data(), G->d_nvec, 3 * nf * 8, cudaMemcpyDeviceToHost));
  if (active) std::memcpy(active, act.data(), nf);
  if (fn) std::memcpy(fn, f.data(), nf * 8);
  if (gap) CK(cudaMemcpy(gap, G->d_gap, nf * 8, cudaMemcpyDeviceToHost));
  if (force) {
    double F[3] = {0, 0, 0};
    for (size_t q = 0; q < nf; ++q)
      if (act[q])
        for (int c = 0; c < 3; ++c) F[c] += f[q] * nv[3 * q + c];
    for (int c = 0; c < 3; ++c) force[c] = F[c];
  }
  return DTT_OK;
}

dtt_status dtt_apply_residual(dtt_grid* G, const double* u, double* p, double* ptilde, double norms[2],
                              int32_t ptr_is_device) {
  if (!G || !u) return fail(DTT_ERR_ARG, "null argument");
  if (!G->mat_set || !G->ref_set) return fail(DTT_ERR_STATE, "material and reference must be set");
  dtt_status st = ensure_ops(G);
  if (st != DTT_OK) return st;
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  // u into op storage (does not touch the solver state)
  double* ud = G->op_d;
  CK(cudaMemcpyAsync(ud, u, n3 * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  float *hi = nullptr, *lo = nullptr;
  if (G->prec == DTT_PREC_MIXED) {
    hi = (float*)G->op_t1;   // reuse: 3NN floats each
    lo = (float*)G->spec;
    CKL(launch_split((long long)n3, ud, hi, lo, s));
  }
  ResidualArgs ra{};
  ra.g = G->g;
  ra.u64 = G->prec == DTT_PREC_FP64 ? ud : nullptr;
  ra.uhi = hi;
  ra.ulo = lo;
  ra.phase = G->phase;
  ra.lam = G->d_lam;
  ra.mu = G->d_mu;
  ra.nphase = G->nphase;
  ra.cmask = nullptr;
  std::memcpy(ra.eps, G->eps, sizeof(ra.eps));
  ra.lam0 = G->lam0;
  ra.mu0 = G->mu0;
  ra.mode = 0;
  ra.pout = G->gbuf;
  ra.xout = G->op_t2;
  ra.partials = G->d_part;
  ra.ctrl = nullptr;
  if (G->prec == DTT_PREC_FP64) CKL(launch_residual<double>(ra, s));
  else CKL(launch_residual<float>(ra, s));
  const int isf = G->prec == DTT_PREC_MIXED;
  auto out = [&](const void* src, double* dst) -> dtt_status {
    CKL(launch_to_double((long long)n3, src, isf, G->op_d, s));
    CK(cudaMemcpyAsync(dst, G->op_d, n3 * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DTT_OK;
  };
  if (p) { st = out(G->gbuf, p); if (st != DTT_OK) return st; }
  if (ptilde) { st = out(G->op_t2, ptilde); if (st != DTT_OK) return st; }
  if (norms) {
    int nb = res_blocks(G);
    std::vector<double> part(RES_STRIDE * (size_t)nb);
    CK(cudaMemcpyAsync(part.data(), G->d_part, part.size() * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double a0 = 0.0, a1 = 0.0;
    for (int b = 0; b < nb; ++b) { a0 += part[RES_STRIDE * b]; a1 += part[RES_STRIDE * b + 1]; }
    norms[0] = a0;
    norms[1] = a1;
  }
  CK(cudaStreamSynchronize(s));
  return DTT_OK;
}

dtt_status dtt_apply_green(dtt_grid* G, const double* ptilde, double* u, int32_t ptr_is_device) {
  if (!G || !ptilde || !u) return fail(DTT_ERR_ARG, "null argument");
  if (!G->ref_set) return fail(DTT_ERR_STATE, "reference not set");
  dtt_status st = ensure_ops(G);
  if (st != DTT_OK) return st;
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  const int isf = G->prec == DTT_PREC_MIXED;
  CK(cudaMemcpyAsync(G->op_d, ptilde, n3 * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CKL(launch_from_double((long long)n3, G->op_d, G->op_t1, isf, s));
  if (isf) st = enqueue_green<float>(G, (const float*)G->op_t1, nullptr, (float*)G->op_t1, (float*)G->op_t2, false, nullptr, 0, 3);
  else st = enqueue_green<double>(G, (const double*)G->op_t1, nullptr, (double*)G->op_t1, (double*)G->op_t2, false, nullptr, 0, 3);
  if (st != DTT_OK) return st;
  CKL(launch_to_double((long long)n3, G->op_t1, isf, G->op_d, s));
  CK(cudaMemcpyAsync(u, G->op_d, n3 * 8, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_tz(G);
}

dtt_status dtt_transform(dtt_grid* G, int32_t component, int32_t inverse, const double* in, double* out,
                         int32_t ptr_is_device) {
  if (!G || !in || !out) return fail(DTT_ERR_ARG, "null argument");
  if (component < 0 || component > 2) return fail(DTT_ERR_ARG, "component in 0..2");
  dtt_status st = ensure_ops(G);
  if (st != DTT_OK) return st;
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  const size_t off = (size_t)component * G->NN;
  const int isf = G->prec == DTT_PREC_MIXED;
  CK(cudaMemsetAsync(G->op_d, 0, n3 * 8, s));
  CK(cudaMemcpyAsync(G->op_d + off, in, (size_t)G->NN * 8,
                     ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CKL(launch_from_double((long long)n3, G->op_d, G->op_t1, isf, s));
  TransformTables tt = tables(G);
  const int axes_f[3] = {0, 1, 2}, axes_i[3] = {2, 1, 0};
  void* a = G->op_t1;
  void* b = G->op_t2;
  for (int q = 0; q < 3; ++q) {
    int ax = inverse ? axes_i[q] : axes_f[q];
    if (isf) CKL(launch_transform_axis<float>(G->g, (const float*)a, (float*)b, tt, ax, inverse, component, 1, nullptr, s));
    else CKL(launch_transform_axis<double>(G->g, (const double*)a, (double*)b, tt, ax, inverse, component, 1, nullptr, s));
    std::swap(a, b);
  }
  CKL(launch_to_double((long long)n3, a, isf, G->op_d, s));
  CK(cudaMemcpyAsync(out, G->op_d + off, (size_t)G->NN * 8,
                     ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DTT_OK;
}

dtt_status dtt_profile_iteration(dtt_grid* G, const dtt_solve_opts* opts, int32_t iters, double* ms) {
  if (!G || !opts || !ms || iters < 1) return fail(DTT_ERR_ARG, "bad argument");
  if (!G->mat_set || !G->ref_set) return fail(DTT_ERR_STATE, "material and reference must be set");
  cudaStream_t s = G->stream;
  // fresh control block that never stops within `iters`
  Ctrl& c = *G->h_ctrl;
  std::memset(&c, 0, sizeof(Ctrl));
  c.max_iter = 1 << 30;
  c.acv_mod = opts->acv_mod > 0 ? opts->acv_mod : 1;
  c.acv_on = opts->acv_on;
  c.contact_on = G->contact ? 1 : 0;
  c.tol = 0.0;
  c.update_tol = 1e-2;
  c.acv_pivot = opts->acv_pivot > 0.0 ? opts->acv_pivot : 1e-14;
  c.no_stop = 1;
  CK(cudaMemcpyAsync(G->d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  cudaEvent_t ev[9];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double acc[9] = {0};
  const bool acv = opts->acv_mod > 0;
  dtt_status st = DTT_OK;
  for (int it = 0; it < iters && st == DTT_OK; ++it) {
    g_prof_ev = ev;
    st = enqueue_iter_any(G, opts->acv_on, acv);
    g_prof_ev = nullptr;
    CK(cudaEventSynchronize(ev[8]));
    for (int k = 0; k < 8; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != DTT_OK) return st;
  // groups: 0 residual [0,1), 1 proj+contact+ctrl [1,2) + [7,8), 2 Anderson [2,3),
  // 3 forward transforms [3,4), 4 Green [4,5), 5 inverse transforms [5,6), 6 increment [6,7)
  ms[0] = acc[0] / iters;
  ms[1] = (acc[1] + acc[7]) / iters;
  ms[2] = acc[2] / iters;
  ms[3] = acc[3] / iters;
  ms[4] = acc[4] / iters;
  ms[5] = acc[5] / iters;
  ms[6] = acc[6] / iters;
  return DTT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free Green step.
//
// Some callers cannot call cudaMalloc while they run: code inside a memory-budgeted
// service that must not grow the device heap after start-up, real-time loops where an
// allocation's implicit synchronisation is unacceptable, or hosts whose allocator is
// owned by another framework.  dtt_apply_green_noalloc lets them apply the Green step to
// their own device buffers without any allocation: the intermediate spectra live in the
// fixed array below, which every GPU that loads this library holds until the process
// exits.  The array's device address is looked up once per device (cudaGetSymbolAddress
// with that device current) on the first call made on that device, so that first call
// should come before any stream capture.  The grid's device must be the current device
// (DTT_ERR_ARG otherwise).  All calls share the array: calls that overlap
// on the GPU (different streams, or different grids used concurrently) race on it.
// Nothing in it has to start at zero: every element a call reads was written earlier
// in the same call.
// ---------------------------------------------------------------------------------------
namespace {

constexpr size_t kGreenScratchBytes = 64ull << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_green_scratch[kGreenScratchBytes];

constexpr int kMaxDevices = 64;
// One address per device; host threads may make their first calls at the same time, so
// the entries are atomics (both would store the same value).
std::atomic<void*> g_green_scratch_addr[kMaxDevices];

// The scratch array's device address on the grid's device.  That device must be the
// current one: the kernels run on the grid's stream, and the symbol lookup below is made
// on the current device.
dtt_status green_scratch_for_grid(const dtt_grid* G, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DTT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != G->device)
    return fail(DTT_ERR_ARG, "the current device (" + std::to_string(dev) + ") is not the grid's device (" +
                                 std::to_string(G->device) + ")");
  if (dev < 0 || dev >= kMaxDevices) return fail(DTT_ERR_ARG, "device ordinal beyond the scratch table");
  void* p = g_green_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    e = cudaGetSymbolAddress(&p, g_green_scratch);
    if (e != cudaSuccess || !p)
      return fail(DTT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_green_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return DTT_OK;
}

}  // namespace

extern "C" dtt_status dtt_apply_green_noalloc(dtt_grid* G, const double* ptilde_dev, double* u_dev) {
  if (!G || !ptilde_dev || !u_dev) return fail(DTT_ERR_ARG, "null argument");
  if (!G->ref_set) return fail(DTT_ERR_STATE, "reference not set");
  const size_t n3 = (size_t)(3 * G->NN);
  const size_t need = n3 * sizeof(double);   // FP64: one work field; mixed: two float fields
  if (need > kGreenScratchBytes)
    return fail(DTT_ERR_ARG, "grid too large for the allocation-free Green step: needs " + std::to_string(need) +
                                 " bytes of scratch, the fixed array holds " + std::to_string(kGreenScratchBytes) +
                                 " (at most " + std::to_string(kGreenScratchBytes / 24) + " nodes)");
  void* scratch = nullptr;
  dtt_status st = green_scratch_for_grid(G, &scratch);
  if (st != DTT_OK) return st;
  cudaStream_t s = G->stream;
  if (G->prec == DTT_PREC_FP64) {
    // in -> scratch -> out ping-pong; the result lands in the caller's output buffer
    st = enqueue_green<double>(G, ptilde_dev, nullptr, u_dev, (double*)scratch, false, nullptr, 0, 3);
    if (st != DTT_OK) return st;
  } else {
    float* a = (float*)scratch;
    float* b = a + n3;
    CKL(launch_from_double((long long)n3, ptilde_dev, a, 1, s));
    st = enqueue_green<float>(G, a, nullptr, a, b, false, nullptr, 0, 3);
    if (st != DTT_OK) return st;
    CKL(launch_to_double((long long)n3, a, 1, u_dev, s));
  }
  CK(cudaStreamSynchronize(s));
  return check_tz(G);
}

// ---------------------------------------------------------------------------------------
// Kernel tuning and batched solves.
//
// A batch of independent cells (many grids of uneven sizes) runs as one CUDA graph whose
// parallel branches are the cells' own iteration sequences, each on the cell's stream:
// small cells fill the GPU together instead of one after another, and one graph launch
// advances every cell by graph_iters iterations.  The tile choices of the two kernels whose
// best shape depends on the grid (the residual kernel's z chunk, the FFT route) are
// measured per grid by dtt_autotune and can be copied to grids of the same size.

namespace {

// Mean milliseconds per iteration of `iters` iterations launched one by one on the grid's
// stream, after one untimed iteration, with a control block that never stops.
dtt_status time_iterations(dtt_grid* G, const dtt_solve_opts* opts, int iters, double* ms) {
  cudaStream_t s = G->stream;
  Ctrl& c = *G->h_ctrl;
  std::memset(&c, 0, sizeof(Ctrl));
  c.max_iter = 1 << 30;
  c.acv_mod = opts->acv_mod > 0 ? opts->acv_mod : 1;
  c.acv_on = opts->acv_on;
  c.contact_on = G->contact ? 1 : 0;
  c.update_tol = 1e-2;
  c.acv_pivot = 1e-14;
  c.no_stop = 1;
  CK(cudaMemcpyAsync(G->d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
  const bool acv = opts->acv_mod > 0;
  dtt_status st = enqueue_iter_any(G, opts->acv_on, acv);
  if (st != DTT_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  for (int k = 0; k < iters && st == DTT_OK; ++k) st = enqueue_iter_any(G, opts->acv_on, acv);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DTT_OK) return st;
  if (e != cudaSuccess) return fail(DTT_ERR_CUDA, std::string("tuning timer: ") + cudaGetErrorString(e));
  *ms = (double)t / iters;
  return DTT_OK;
}

// u~, the rings and the step back to zero (state after tuning runs).
dtt_status reset_state(dtt_grid* G) {
  cudaStream_t s = G->stream;
  const size_t n3 = (size_t)(3 * G->NN);
  if (G->u64) CK(cudaMemsetAsync(G->u64, 0, n3 * 8, s));
  if (G->uhi) CK(cudaMemsetAsync(G->uhi, 0, n3 * 4, s));
  if (G->ulo) CK(cudaMemsetAsync(G->ulo, 0, n3 * 4, s));
  for (int k = 0; k < 5; ++k) CK(cudaMemsetAsync(G->S[k], 0, n3 * G->esz, s));
  for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(G->R[k], 0, n3 * G->esz, s));
  for (int k = 0; k < 4; ++k) CK(cudaMemsetAsync(G->Gr[k], 0, n3 * G->esz, s));
  // the Green-input ring points at the own buffers again (a solve may leave aliases of p)
  CK(cudaMemcpyAsync(G->d_Gring, G->d_Gown, 4 * sizeof(void*), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(G->step, 0, n3 * G->esz, s));
  CK(cudaStreamSynchronize(s));
  return DTT_OK;
}

dtt_status apply_tiling(dtt_grid* G, int zc, int generic, int z_route, int warp) {
  G->g.zc_override = zc;
  G->g.fft_generic = generic;
  G->z_route = (z_route == 1 && G->tz_ok) ? 1 : 0;
  G->fft_warp = warp ? 1 : 0;
  invalidate_graph(G);
  return ensure_partials(G);
}

struct BatchCache {
  std::vector<unsigned long long> key;   // device, opts key, then (id, version) per cell
  cudaGraphExec_t exec = nullptr;
  bool looped = false;                   // exec runs the whole batch (conditional WHILE node)
  int* d_rounds = nullptr;
  cudaStream_t bs = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  Ctrl** d_ctrls = nullptr;
  int* d_done = nullptr;
  int* h_done = nullptr;
  int cap = 0;
};
BatchCache g_batch;

dtt_status batch_buffers(int n) {
  if (!g_batch.bs) CK(cudaStreamCreateWithFlags(&g_batch.bs, cudaStreamNonBlocking));
  if (!g_batch.d_rounds) CK(cudaMalloc(&g_batch.d_rounds, 2 * sizeof(int)));
  if (!g_batch.fork) CK(cudaEventCreateWithFlags(&g_batch.fork, cudaEventDisableTiming));
  if (!g_batch.join) CK(cudaEventCreateWithFlags(&g_batch.join, cudaEventDisableTiming));
  if (n > g_batch.cap) {
    if (g_batch.d_ctrls) cudaFree(g_batch.d_ctrls);
    if (g_batch.d_done) cudaFree(g_batch.d_done);
    if (g_batch.h_done) cudaFreeHost(g_batch.h_done);
    g_batch.d_ctrls = nullptr;
    g_batch.d_done = nullptr;
    g_batch.h_done = nullptr;
    g_batch.cap = 0;
    CK(cudaMalloc(&g_batch.d_ctrls, n * sizeof(Ctrl*)));
    CK(cudaMalloc(&g_batch.d_done, n * sizeof(int)));
    CK(cudaMallocHost(&g_batch.h_done, n * sizeof(int)));
    g_batch.cap = n;
  }
  return DTT_OK;
}

}  // namespace

extern "C" {

dtt_status dtt_autotune(dtt_grid* G, const dtt_solve_opts* opts, int32_t iters, dtt_tuning* best) {
  dtt_status st = check_solve(G, opts);
  if (st != DTT_OK) return st;
  if (iters < 1) return fail(DTT_ERR_ARG, "iters must be >= 1");
  double t_best = 1e300;
  int zc_best = 0, gen_best = 0, zr_best = 0, wp_best = 0;
  // the warp-register sweeps (where the grid allows them), then the Stockham routes
  const bool warp_ok = G->prec == DTT_PREC_MIXED && wfft_supported(G->g, tables(G));
  for (int wp = (warp_ok ? 1 : 0); wp >= 0; --wp)
    for (int zr = 0; zr < ((G->tz_ok && !wp) ? 2 : 1); ++zr)
      for (int gen = 0; gen < (wp ? 1 : 2); ++gen) {
        if ((st = apply_tiling(G, 0, gen, zr, wp)) != DTT_OK) return st;
        double t = 0.0;
        if ((st = time_iterations(G, opts, iters, &t)) != DTT_OK) return st;
        if (t < t_best) { t_best = t; gen_best = gen; zr_best = zr; wp_best = wp; }
      }
  const int zcs[6] = {2, 4, 8, 16, 32, 64};
  for (int q = 0; q < 6; ++q) {
    if (zcs[q] > 2 * G->g.nn[2]) break;
    if ((st = apply_tiling(G, zcs[q], gen_best, zr_best, wp_best)) != DTT_OK) return st;
    double t = 0.0;
    if ((st = time_iterations(G, opts, iters, &t)) != DTT_OK) return st;
    if (t < t_best) { t_best = t; zc_best = zcs[q]; }
  }
  if ((st = apply_tiling(G, zc_best, gen_best, zr_best, wp_best)) != DTT_OK) return st;
  if ((st = reset_state(G)) != DTT_OK) return st;
  if ((st = check_tz(G)) != DTT_OK) return st;
  if (best) {
    best->residual_zchunk = zc_best;
    best->fft_generic = gen_best;
    best->z_route = zr_best;
    best->fft_warp = wp_best;
    best->ms_per_iteration = t_best;
  }
  return DTT_OK;
}

dtt_status dtt_set_tuning(dtt_grid* G, const dtt_tuning* t) {
  if (!G || !t) return fail(DTT_ERR_ARG, "null argument");
  if (t->residual_zchunk != 0 && (t->residual_zchunk < 2 || t->residual_zchunk > 64))
    return fail(DTT_ERR_ARG, "residual_zchunk must be 0 or in [2, 64]");
  if (t->fft_generic != 0 && t->fft_generic != 1) return fail(DTT_ERR_ARG, "fft_generic must be 0 or 1");
  if (t->z_route != 0 && t->z_route != 1) return fail(DTT_ERR_ARG, "z_route must be 0 or 1");
  if (t->z_route == 1 && !G->tz_ok)
    return fail(DTT_ERR_ARG, "z_route 1 needs a mixed-precision grid whose z operand has at most 256 nodes");
  if (t->fft_warp != 0 && t->fft_warp != 1) return fail(DTT_ERR_ARG, "fft_warp must be 0 or 1");
  return apply_tiling(G, t->residual_zchunk, t->fft_generic, t->z_route, t->fft_warp);
}

dtt_status dtt_batch_solve(int32_t ncell, dtt_grid* const* cells, const dtt_solve_opts* opts, dtt_report* reports) {
  if (ncell < 1 || !cells || !opts) return fail(DTT_ERR_ARG, "ncell >= 1, cells and opts required");
  for (int i = 0; i < ncell; ++i) {
    dtt_status st = check_solve(cells[i], opts);
    if (st != DTT_OK) return st;
    for (int j = 0; j < i; ++j)
      if (cells[j] == cells[i]) return fail(DTT_ERR_ARG, "a grid appears twice in the batch");
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < ncell; ++i) {
    dtt_status st = prepare_solve(cells[i], opts);
    if (st != DTT_OK) return st;
    CK(cudaStreamSynchronize(cells[i]->stream));
  }
  dtt_status st = batch_buffers(ncell);
  if (st != DTT_OK) return st;
  const bool acv = opts->acv_mod > 0;
  const int iters = graph_iters_of(opts);
  std::vector<unsigned long long> key;
  key.push_back((unsigned long long)dev);
  key.push_back((unsigned long long)graph_key_of(opts));
  for (int i = 0; i < ncell; ++i) {
    key.push_back(cells[i]->id);
    key.push_back(cells[i]->version);
  }
  cudaStream_t bs = g_batch.bs;
  if (!g_batch.exec || key != g_batch.key) {
    if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
    g_batch.exec = nullptr;
    g_batch.key.clear();
    std::vector<Ctrl*> ctrls(ncell);
    for (int i = 0; i < ncell; ++i) ctrls[i] = cells[i]->d_ctrl;
    CK(cudaMemcpy(g_batch.d_ctrls, ctrls.data(), ncell * sizeof(Ctrl*), cudaMemcpyHostToDevice));
    // fork-join round: every cell's iterations on its own stream, joined back to bs
    auto round = [&]() {
      dtt_status rs = DTT_OK;
      cudaEventRecord(g_batch.fork, bs);
      for (int i = 0; i < ncell; ++i) {
        cudaStreamWaitEvent(cells[i]->stream, g_batch.fork, 0);
        for (int k = 0; k < iters && rs == DTT_OK; ++k) rs = enqueue_iter_any(cells[i], opts->acv_on, acv);
        cudaEventRecord(g_batch.join, cells[i]->stream);
        cudaStreamWaitEvent(bs, g_batch.join, 0);
        if (rs != DTT_OK) break;
      }
      return rs;
    };
    // the whole batch as one launch (conditional WHILE node), else one round per launch
    bool looped = false;
    st = build_loop_graph(bs, round, g_batch.d_ctrls, nullptr, ncell, g_batch.d_rounds, &g_batch.exec, &looped);
    if (st != DTT_OK) return st;
    g_batch.looped = looped;
    if (!looped) {
      CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
      st = round();
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(bs, &graph);
      if (st != DTT_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st != DTT_OK) return st;
        return fail(DTT_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&g_batch.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g_batch.exec = nullptr;
        return fail(DTT_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    g_batch.key = key;
  }
  long long launched = 0;
  const long long cap = (long long)opts->max_iter + 2LL * iters + 8;
  if (g_batch.looped) {
    if ((st = arm_loop(g_batch.d_rounds, (int)std::min<long long>(cap / iters + 2, 1 << 30), bs)) != DTT_OK) return st;
    CK(cudaGraphLaunch(g_batch.exec, bs));
    CK(cudaStreamSynchronize(bs));
  }
  while (!g_batch.looped) {
    CK(cudaGraphLaunch(g_batch.exec, bs));
    launched += iters;
    CKL(launch_batch_done(g_batch.d_ctrls, ncell, g_batch.d_done, bs));
    CK(cudaMemcpyAsync(g_batch.h_done, g_batch.d_done, ncell * sizeof(int), cudaMemcpyDeviceToHost, bs));
    CK(cudaStreamSynchronize(bs));
    bool all = true;
    for (int i = 0; i < ncell && all; ++i) all = g_batch.h_done[i] != 0;
    if (all || launched > cap) break;   // the cap cannot be reached: cells stop at max_iter
  }
  dtt_status first = DTT_OK;
  for (int i = 0; i < ncell; ++i) {
    dtt_status si = finish_solve(cells[i], t0, reports ? &reports[i] : nullptr);
    if (si != DTT_OK && first == DTT_OK) first = si;
  }
  return first;
}

}  // extern "C"

// Host side of the warm-start network (include/dtt_net.h): parameters, workspace, the
// forward and backward sequences of kernel launches, Adam, and the C entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "dtt_net.h"
#include "grid_internal.cuh"
#include "net_internal.cuh"

using namespace dtt;
using namespace dtt::net;
using bf16 = __nv_bfloat16;

namespace {

#define NCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return set_error(DTT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define NCKL(rc)                                                                            \
  do {                                                                                      \
    int r_ = (rc);                                                                          \
    if (r_ != 0) return set_error(DTT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString((cudaError_t)r_)); \
  } while (0)

constexpr int NLAYER = 11;

struct Layer {
  int cin, cout;
  long long woff, boff;   // offsets of W and b in the packed parameter vector
  bf16* wt;               // [27][cout][cin]
  bf16* wd;               // [27][cin][cout]
};

struct Dims {
  int n[3];
  long long V() const { return (long long)n[0] * n[1] * n[2]; }
};

Dims half(const Dims& d) { return Dims{{(d.n[0] + 1) / 2, (d.n[1] + 1) / 2, (d.n[2] + 1) / 2}}; }

}  // namespace

struct dtt_net {
  int c1 = 16, c2 = 32, c3 = 64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Layer L[NLAYER]{};
  long long np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16* wbuf = nullptr;
  int step = 0;
  float grad_weight = 0.f;   // weight of the difference term of the loss
  // workspace (capacities in voxels per level)
  long long cap0 = 0, cap1 = 0, cap2 = 0;
  Dims d0{}, d1{}, d2{};
  float* xf = nullptr;   // [V0][16] features (FP32)
  bf16* x = nullptr;     // [V0][16]
  bf16 *a0 = nullptr, *e1 = nullptr, *p1 = nullptr, *a2 = nullptr, *e2 = nullptr, *p2 = nullptr, *a4 = nullptr,
       *e3 = nullptr, *u2 = nullptr, *r6 = nullptr, *d2a = nullptr, *d2b = nullptr, *u1 = nullptr, *r8 = nullptr,
       *d1a = nullptr, *d1b = nullptr;
  float* y = nullptr;    // [V0][16]
  float* tgt = nullptr;  // [V0][3]
  float *gP = nullptr, *gQ = nullptr, *ge1 = nullptr, *ge2 = nullptr;
  bf16* dz = nullptr;
  double* d_loss = nullptr;
  double* d_u = nullptr;   // [3][V0] guess of u~ (float64)
  float* d_en = nullptr;   // per-phase normalised stiffness
  // increment mode
  float* inc_t = nullptr;  // [V0][4] targets
  float* inc_m = nullptr;  // [V0] surface mask of the pressure term
  float* d_fmax = nullptr; // largest contact pressure of the previous increment
  uint8_t* d_act = nullptr;
  int act_cap = 0;
  float inc_wp = 1.f;      // weight of the pressure term of the loss
  float inc_thr = 0.05f;   // predicted pressure above which a surface node starts in contact
  int win_lat = 0;         // window: nodes across the contact face (0: whole grid)
  int win_dep = 0;         // window: node layers below the contact face (0: whole grid)
  double* d_ug = nullptr;  // [3][NN] guess of u~ on the whole grid (increment mode)
  long long ug_cap = 0;
  // tracing (dtt_net_layer_trace): the input activation and the output gradient through the
  // ReLU of one layer, copied by its backward pass
  int trace_layer = -1;
  bf16* tr_in = nullptr;
  bf16* tr_dz = nullptr;
  float* tr_dx = nullptr;
};

namespace {

template <typename P>
dtt_status nalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return DTT_OK;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? DTT_ERR_OOM : DTT_ERR_CUDA,
                     std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return DTT_OK;
}
template <typename P>
void nfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void free_workspace(dtt_net* N) {
  nfree(N->xf); nfree(N->x); nfree(N->a0); nfree(N->e1); nfree(N->p1); nfree(N->a2); nfree(N->e2); nfree(N->p2);
  nfree(N->a4); nfree(N->e3); nfree(N->u2); nfree(N->r6); nfree(N->d2a); nfree(N->d2b); nfree(N->u1); nfree(N->r8);
  nfree(N->d1a); nfree(N->d1b); nfree(N->y); nfree(N->tgt); nfree(N->gP); nfree(N->gQ); nfree(N->ge1); nfree(N->ge2);
  nfree(N->dz); nfree(N->d_u); nfree(N->inc_t); nfree(N->inc_m);
  N->cap0 = N->cap1 = N->cap2 = 0;
}

// Workspace for a grid of nx x ny x nz nodes (kept while later grids fit in it).
dtt_status ensure_workspace(dtt_net* N, int nx, int ny, int nz) {
  N->d0 = Dims{{nx, ny, nz}};
  N->d1 = half(N->d0);
  N->d2 = half(N->d1);
  const long long V0 = N->d0.V(), V1 = N->d1.V(), V2 = N->d2.V();
  if (V0 <= N->cap0 && V1 <= N->cap1 && V2 <= N->cap2) return DTT_OK;
  free_workspace(N);
  const long long c0 = std::max(V0, 1LL), cc1 = std::max(V1, 1LL), cc2 = std::max(V2, 1LL);
  const int c1 = N->c1, c2 = N->c2, c3 = N->c3;
  const int cmax = std::max(std::max(c1, c2), std::max(c3, 16));
  dtt_status s = DTT_OK;
  auto B = [&](bf16** p, long long n) { if (s == DTT_OK) s = nalloc(p, (size_t)n * sizeof(bf16)); };
  auto F = [&](float** p, long long n) { if (s == DTT_OK) s = nalloc(p, (size_t)n * sizeof(float)); };
  F(&N->xf, c0 * 16); B(&N->x, c0 * 16);
  B(&N->a0, c0 * c1); B(&N->e1, c0 * c1); B(&N->p1, cc1 * c1); B(&N->a2, cc1 * c2); B(&N->e2, cc1 * c2);
  B(&N->p2, cc2 * c2); B(&N->a4, cc2 * c3); B(&N->e3, cc2 * c3); B(&N->u2, cc1 * c3); B(&N->r6, cc1 * c2);
  B(&N->d2a, cc1 * c2); B(&N->d2b, cc1 * c2); B(&N->u1, c0 * c2); B(&N->r8, c0 * c1); B(&N->d1a, c0 * c1);
  B(&N->d1b, c0 * c1);
  F(&N->y, c0 * NET_COUT); F(&N->tgt, c0 * 3);
  F(&N->gP, c0 * cmax); F(&N->gQ, c0 * cmax); F(&N->ge1, c0 * c1); F(&N->ge2, cc1 * c2);
  B(&N->dz, c0 * cmax);
  F(&N->inc_t, c0 * 4); F(&N->inc_m, c0);
  if (s == DTT_OK) s = nalloc(&N->d_u, (size_t)c0 * 3 * sizeof(double));
  if (s != DTT_OK) {
    free_workspace(N);
    return s;
  }
  N->cap0 = c0;
  N->cap1 = cc1;
  N->cap2 = cc2;
  return DTT_OK;
}

dtt_status refresh_bf16(dtt_net* N) {
  for (int l = 0; l < NLAYER; ++l)
    NCKL(launch_relayout(N->p + N->L[l].woff, N->L[l].cin, N->L[l].cout, N->L[l].wt, N->L[l].wd, N->stream));
  return DTT_OK;
}

}  // namespace

namespace {

ConvArgs conv_args(const dtt_net* N, int l, const Dims& d) {
  ConvArgs a{};
  a.cin = N->L[l].cin;
  a.cout = N->L[l].cout;
  a.nx = d.n[0];
  a.ny = d.n[1];
  a.nz = d.n[2];
  a.wt = N->L[l].wt;
  a.wd = N->L[l].wd;
  a.bias = N->p + N->L[l].boff;
  a.dw = N->g + N->L[l].woff;
  a.db = N->g + N->L[l].boff;
  return a;
}

dtt_status fwd_layer(dtt_net* N, int l, const Dims& d, const bf16* in, bf16* out, int flags,
                     const bf16* skip = nullptr, bf16* r = nullptr, float* outf = nullptr) {
  ConvArgs a = conv_args(N, l, d);
  a.flags = flags;
  a.x = in;
  a.y = out;
  a.yf = outf;
  a.skip = skip;
  a.r = r;
  NCKL(launch_conv_fwd(a, N->stream));
  return DTT_OK;
}

// gradient G (FP32, at the layer's output) -> dZ through the layer's ReLU (R = its ReLU
// output, null for the linear last layer), then weight/bias gradients and dX
dtt_status bwd_layer(dtt_net* N, int l, const Dims& d, const bf16* in, const float* G, const bf16* R, float* dX) {
  ConvArgs a = conv_args(N, l, d);
  NCKL(launch_relu_bwd(G, R, d.V() * a.cout, N->dz, N->stream));
  if (l == N->trace_layer && N->tr_in && N->tr_dz) {
    NCK(cudaMemcpyAsync(N->tr_in, in, (size_t)d.V() * a.cin * sizeof(bf16), cudaMemcpyDeviceToDevice, N->stream));
    NCK(cudaMemcpyAsync(N->tr_dz, N->dz, (size_t)d.V() * a.cout * sizeof(bf16), cudaMemcpyDeviceToDevice, N->stream));
  }
  a.x = in;
  a.dz = N->dz;
  a.dx = dX;
  NCKL(launch_conv_bwd(a, N->stream));
  if (l == N->trace_layer && N->tr_dx && dX)
    NCK(cudaMemcpyAsync(N->tr_dx, dX, (size_t)d.V() * a.cin * sizeof(float), cudaMemcpyDeviceToDevice, N->stream));
  return DTT_OK;
}

// forward pass from N->x (BF16 features) to N->y (FP32)
dtt_status forward(dtt_net* N) {
  const Dims &d0 = N->d0, &d1 = N->d1, &d2 = N->d2;
  cudaStream_t s = N->stream;
  dtt_status st;
  if ((st = fwd_layer(N, 0, d0, N->x, N->a0, CF_RELU)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 1, d0, N->a0, N->e1, CF_RELU)) != DTT_OK) return st;
  NCKL(launch_pool_fwd(N->e1, d0.n[0], d0.n[1], d0.n[2], N->c1, N->p1, s));
  if ((st = fwd_layer(N, 2, d1, N->p1, N->a2, CF_RELU)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 3, d1, N->a2, N->e2, CF_RELU)) != DTT_OK) return st;
  NCKL(launch_pool_fwd(N->e2, d1.n[0], d1.n[1], d1.n[2], N->c2, N->p2, s));
  if ((st = fwd_layer(N, 4, d2, N->p2, N->a4, CF_RELU)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 5, d2, N->a4, N->e3, CF_RELU)) != DTT_OK) return st;
  NCKL(launch_up_fwd(N->e3, d1.n[0], d1.n[1], d1.n[2], N->c3, N->u2, s));
  if ((st = fwd_layer(N, 6, d1, N->u2, N->d2a, CF_RELU | CF_SKIP, N->e2, N->r6)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 7, d1, N->d2a, N->d2b, CF_RELU)) != DTT_OK) return st;
  NCKL(launch_up_fwd(N->d2b, d0.n[0], d0.n[1], d0.n[2], N->c2, N->u1, s));
  if ((st = fwd_layer(N, 8, d0, N->u1, N->d1a, CF_RELU | CF_SKIP, N->e1, N->r8)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 9, d0, N->d1a, N->d1b, CF_RELU)) != DTT_OK) return st;
  if ((st = fwd_layer(N, 10, d0, N->d1b, nullptr, CF_F32, nullptr, nullptr, N->y)) != DTT_OK) return st;
  return DTT_OK;
}

dtt_status bwd_chain(dtt_net* N);

// loss against N->tgt and the gradients of every parameter into N->g
dtt_status backward(dtt_net* N, double* loss) {
  const Dims& d0 = N->d0;
  cudaStream_t s = N->stream;
  NCK(cudaMemsetAsync(N->g, 0, (size_t)N->np * sizeof(float), s));
  NCK(cudaMemsetAsync(N->d_loss, 0, sizeof(double), s));
  const float sc = (float)std::max(d0.n[0], std::max(d0.n[1], d0.n[2]));
  NCKL(launch_loss(N->y, N->tgt, d0.n[0], d0.n[1], d0.n[2], NET_COUT, N->grad_weight * sc * sc, N->gP, N->d_loss, s));
  dtt_status st = bwd_chain(N);
  if (st != DTT_OK) return st;
  if (loss) {
    NCK(cudaMemcpyAsync(loss, N->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
  }
  return DTT_OK;
}

// the layers' backward passes from the output gradient in N->gP (parameter gradients
// accumulate into N->g, which the caller has cleared)
dtt_status bwd_chain(dtt_net* N) {
  const Dims &d0 = N->d0, &d1 = N->d1, &d2 = N->d2;
  cudaStream_t s = N->stream;
  const int c1 = N->c1, c2 = N->c2, c3 = N->c3;
  (void)c3;
  dtt_status st;
  if ((st = bwd_layer(N, 10, d0, N->d1b, N->gP, nullptr, N->gQ)) != DTT_OK) return st;
  if ((st = bwd_layer(N, 9, d0, N->d1a, N->gQ, N->d1b, N->gP)) != DTT_OK) return st;
  NCK(cudaMemcpyAsync(N->ge1, N->gP, (size_t)d0.V() * c1 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if ((st = bwd_layer(N, 8, d0, N->u1, N->gP, N->r8, N->gQ)) != DTT_OK) return st;
  NCKL(launch_up_bwd(N->gQ, d0.n[0], d0.n[1], d0.n[2], c2, N->gP, s));
  if ((st = bwd_layer(N, 7, d1, N->d2a, N->gP, N->d2b, N->gQ)) != DTT_OK) return st;
  NCK(cudaMemcpyAsync(N->ge2, N->gQ, (size_t)d1.V() * c2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if ((st = bwd_layer(N, 6, d1, N->u2, N->gQ, N->r6, N->gP)) != DTT_OK) return st;
  NCKL(launch_up_bwd(N->gP, d1.n[0], d1.n[1], d1.n[2], c3, N->gQ, s));
  if ((st = bwd_layer(N, 5, d2, N->a4, N->gQ, N->e3, N->gP)) != DTT_OK) return st;
  if ((st = bwd_layer(N, 4, d2, N->p2, N->gP, N->a4, N->gQ)) != DTT_OK) return st;
  NCKL(launch_pool_bwd_add(N->gQ, d1.n[0], d1.n[1], d1.n[2], c2, N->ge2, s));
  if ((st = bwd_layer(N, 3, d1, N->a2, N->ge2, N->e2, N->gP)) != DTT_OK) return st;
  if ((st = bwd_layer(N, 2, d1, N->p1, N->gP, N->a2, N->gQ)) != DTT_OK) return st;
  NCKL(launch_pool_bwd_add(N->gQ, d0.n[0], d0.n[1], d0.n[2], c1, N->ge1, s));
  if ((st = bwd_layer(N, 1, d0, N->a0, N->ge1, N->e1, N->gP)) != DTT_OK) return st;
  if ((st = bwd_layer(N, 0, d0, N->x, N->gP, N->a0, nullptr)) != DTT_OK) return st;
  return DTT_OK;
}

dtt_status upload_input(dtt_net* N, const float* x_host) {
  const long long V = N->d0.V();
  NCK(cudaMemcpyAsync(N->xf, x_host, (size_t)V * 16 * sizeof(float), cudaMemcpyHostToDevice, N->stream));
  NCKL(launch_f2bf(N->xf, V * 16, N->x, N->stream));
  return DTT_OK;
}

Window whole_grid(const dtt_grid* G) {
  Window w{};
  for (int d = 0; d < 3; ++d) {
    w.o[d] = 0;
    w.n[d] = G->g.nn[d];
  }
  return w;
}

// features of a grid's nodes inside window w into N->xf / N->x (workspace sized for w)
dtt_status grid_features(dtt_net* N, dtt_grid* G, const Window& w) {
  if (!G->mat_set) return set_error(DTT_ERR_STATE, "dtt_set_material not called");
  dtt_status st = ensure_workspace(N, w.n[0], w.n[1], w.n[2]);
  if (st != DTT_OK) return st;
  std::vector<double> lam(G->nphase), mu(G->nphase);
  NCK(cudaMemcpy(lam.data(), G->d_lam, G->nphase * sizeof(double), cudaMemcpyDeviceToHost));
  NCK(cudaMemcpy(mu.data(), G->d_mu, G->nphase * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<float> en(MAX_PHASE, 0.f);
  double emax = 0.0;
  std::vector<double> E(G->nphase);
  for (int q = 0; q < G->nphase; ++q) {
    E[q] = (lam[q] + mu[q] > 0.0) ? mu[q] * (3.0 * lam[q] + 2.0 * mu[q]) / (lam[q] + mu[q]) : 0.0;
    emax = std::max(emax, E[q]);
  }
  for (int q = 0; q < G->nphase; ++q) en[q] = emax > 0.0 ? (float)(E[q] / emax) : 0.f;
  if (!N->d_en) {
    st = nalloc(&N->d_en, MAX_PHASE * sizeof(float));
    if (st != DTT_OK) return st;
  }
  NCK(cudaMemcpyAsync(N->d_en, en.data(), MAX_PHASE * sizeof(float), cudaMemcpyHostToDevice, N->stream));
  FeatArgs fa{};
  fa.g = G->g;
  fa.w = w;
  fa.phase = G->phase;
  fa.enorm = N->d_en;
  fa.cmask = G->cmask;
  const double e6[6] = {G->eps[0][0], G->eps[1][1], G->eps[2][2], G->eps[1][2], G->eps[0][2], G->eps[0][1]};
  for (int q = 0; q < 6; ++q) fa.eps6[q] = (float)(1000.0 * e6[q]);
  fa.x = N->xf;
  NCKL(launch_features(fa, N->stream));
  NCKL(launch_f2bf(N->xf, N->d0.V() * 16, N->x, N->stream));
  return DTT_OK;
}

// Increment mode: base features of the grid, then the increment channels (secant
// prediction, surface gap at the moved sphere, previous pressure) from u~ of increment
// k-1 (the grid's current u~), u~ of increment k-2 (u2, device, null = zero), the previous
// normal reactions fn_prev (device, per surface node) and the depths d_(k-2), d_(k-1), d_k.
dtt_status inc_setup(dtt_net* N, dtt_grid* G, const double* u2, const double* fn_prev, const double depth[3],
                     IncArgs& a) {
  if (!G->contact) return set_error(DTT_ERR_STATE, "no indenter set");
  if (!depth) return set_error(DTT_ERR_ARG, "null argument");
  if (!(depth[0] >= 0.0) || !(depth[1] > depth[0]) || !(depth[2] > depth[1]))
    return set_error(DTT_ERR_ARG, "depths must satisfy 0 <= d_(k-2) < d_(k-1) < d_k");
  // the window: win_dep layers from the contact face inward, win_lat nodes across it
  // centred under the sphere
  Window w = whole_grid(G);
  for (int d = 0; d < 3; ++d) {
    const int nn = G->g.nn[d];
    if (d == G->c_axis) {
      if (N->win_dep > 0 && N->win_dep < nn) {
        w.n[d] = N->win_dep;
        w.o[d] = G->c_face == 1 ? nn - N->win_dep : 0;
      }
    } else if (N->win_lat > 0 && N->win_lat < nn) {
      w.n[d] = N->win_lat;
      const int c = (int)std::lround(G->center[d] / G->g.h) - N->win_lat / 2;
      w.o[d] = std::min(std::max(c, 0), nn - N->win_lat);
    }
  }
  dtt_status st = grid_features(N, G, w);
  if (st != DTT_OK) return st;
  if (!N->d_fmax && (st = nalloc(&N->d_fmax, sizeof(float))) != DTT_OK) return st;
  const double p0 = std::pow(depth[0], 1.5), p1 = std::pow(depth[1], 1.5), p2 = std::pow(depth[2], 1.5);
  a = IncArgs{};
  a.g = G->g;
  a.w = w;
  a.u64 = G->u64;
  a.uhi = G->uhi;
  a.ulo = G->ulo;
  a.u2 = u2;
  a.s_sec = (p2 - p1) / (p1 - p0);
  a.dd = depth[2] - depth[1];
  a.nface = G->nface;
  a.node = G->d_face;
  // fn_prev = NULL: the grid's reactions of its last solve on that solve's contact set
  a.fn_prev = fn_prev ? fn_prev : G->d_fn;
  a.fn_act = fn_prev ? nullptr : G->d_active;
  for (int c = 0; c < 3; ++c) a.center[c] = G->center[c];
  a.radius = G->radius;
  std::memcpy(a.eps, G->eps, sizeof(a.eps));
  a.fmax = N->d_fmax;
  a.x = N->xf;
  NCKL(launch_inc_fmax(a, N->stream));
  NCKL(launch_inc_features(a, N->stream));
  NCKL(launch_f2bf(N->xf, N->d0.V() * 16, N->x, N->stream));
  return DTT_OK;
}

double u_scale(const dtt_grid* G) {
  const int nmax = std::max(G->g.nvox[0], std::max(G->g.nvox[1], G->g.nvox[2]));
  return 1e-3 * nmax;
}

}  // namespace

namespace {
// Features, target, forward pass, loss and backward pass of one cell (the gradient in N->g,
// the loss on the host).
dtt_status cell_loss_grad(dtt_net* N, dtt_grid* G, const double* u_target, double* loss) {
  dtt_status s = grid_features(N, G, whole_grid(G));
  if (s != DTT_OK) return s;
  const long long V = N->d0.V();
  const double inv = 1.0 / u_scale(G);
  std::vector<float> t((size_t)V * 3);
  for (int c = 0; c < 3; ++c)
    for (long long v = 0; v < V; ++v) t[v * 3 + c] = (float)(u_target[c * V + v] * inv);
  NCK(cudaMemcpyAsync(N->tgt, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, N->stream));
  if ((s = forward(N)) != DTT_OK) return s;
  return backward(N, loss);
}

dtt_status check_device_floats(const float* p, long long n, const char* what);
}  // namespace

extern "C" {

dtt_status dtt_net_create(dtt_net** out, int32_t c1, int32_t c2, int32_t c3, uint64_t seed, void* stream) {
  if (!out) return set_error(DTT_ERR_ARG, "null output");
  *out = nullptr;
  for (int c : {c1, c2, c3})
    if (c != 16 && c != 32 && c != 64) return set_error(DTT_ERR_ARG, "channel counts must be 16, 32 or 64");
  dtt_net* N = new dtt_net();
  N->c1 = c1;
  N->c2 = c2;
  N->c3 = c3;
  if (stream) {
    N->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&N->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete N;
      return set_error(DTT_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    N->own_stream = true;
  }
  const int io[NLAYER][2] = {{NET_CIN, c1}, {c1, c1}, {c1, c2}, {c2, c2}, {c2, c3}, {c3, c3},
                             {c3, c2},      {c2, c2}, {c2, c1}, {c1, c1}, {c1, NET_COUT}};
  long long off = 0, wb = 0;
  for (int l = 0; l < NLAYER; ++l) {
    N->L[l].cin = io[l][0];
    N->L[l].cout = io[l][1];
    N->L[l].woff = off;
    off += 27LL * io[l][0] * io[l][1];
    N->L[l].boff = off;
    off += io[l][1];
    wb += 27LL * io[l][0] * io[l][1];
  }
  N->np = off;
  dtt_status s = nalloc(&N->p, N->np * sizeof(float));
  if (s == DTT_OK) s = nalloc(&N->g, N->np * sizeof(float));
  if (s == DTT_OK) s = nalloc(&N->m, N->np * sizeof(float));
  if (s == DTT_OK) s = nalloc(&N->v, N->np * sizeof(float));
  if (s == DTT_OK) s = nalloc(&N->wbuf, 2 * wb * sizeof(bf16));
  if (s == DTT_OK) s = nalloc(&N->d_loss, sizeof(double));
  if (s != DTT_OK) {
    dtt_net_destroy(N);
    return s;
  }
  long long wo = 0;
  for (int l = 0; l < NLAYER; ++l) {
    const long long n = 27LL * N->L[l].cin * N->L[l].cout;
    N->L[l].wt = N->wbuf + wo;
    N->L[l].wd = N->wbuf + wb + wo;
    wo += n;
  }
  // He-normal weights, zero biases
  std::vector<float> h(N->np, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < NLAYER; ++l) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (27.f * N->L[l].cin)));
    const long long n = 27LL * N->L[l].cin * N->L[l].cout;
    for (long long q = 0; q < n; ++q) h[N->L[l].woff + q] = nd(rng);
  }
  s = dtt_net_set_params(N, h.data());
  if (s != DTT_OK) {
    dtt_net_destroy(N);
    return s;
  }
  *out = N;
  return DTT_OK;
}

void dtt_net_destroy(dtt_net* N) {
  if (!N) return;
  if (N->stream) cudaStreamSynchronize(N->stream);
  free_workspace(N);
  nfree(N->p);
  nfree(N->g);
  nfree(N->m);
  nfree(N->v);
  nfree(N->wbuf);
  nfree(N->d_loss);
  nfree(N->d_en);
  nfree(N->d_fmax);
  nfree(N->d_act);
  nfree(N->d_ug);
  if (N->own_stream && N->stream) cudaStreamDestroy(N->stream);
  delete N;
}

int64_t dtt_net_num_params(const dtt_net* N) { return N ? N->np : 0; }

dtt_status dtt_net_set_loss(dtt_net* N, float grad_weight) {
  if (!N || !(grad_weight >= 0.f)) return set_error(DTT_ERR_ARG, "grad_weight must be >= 0");
  N->grad_weight = grad_weight;
  return DTT_OK;
}

dtt_status dtt_net_get_params(const dtt_net* N, float* params) {
  if (!N || !params) return set_error(DTT_ERR_ARG, "null argument");
  NCK(cudaMemcpyAsync(params, N->p, N->np * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  return DTT_OK;
}

dtt_status dtt_net_set_params(dtt_net* N, const float* params) {
  if (!N || !params) return set_error(DTT_ERR_ARG, "null argument");
  NCK(cudaMemcpyAsync(N->p, params, N->np * sizeof(float), cudaMemcpyHostToDevice, N->stream));
  NCK(cudaMemsetAsync(N->m, 0, N->np * sizeof(float), N->stream));
  NCK(cudaMemsetAsync(N->v, 0, N->np * sizeof(float), N->stream));
  N->step = 0;
  dtt_status s = refresh_bf16(N);
  if (s != DTT_OK) return s;
  NCK(cudaStreamSynchronize(N->stream));
  return DTT_OK;
}

dtt_status dtt_net_loss_grad(dtt_net* N, int32_t nx, int32_t ny, int32_t nz, const float* x, const float* target,
                             double* loss, float* grad) {
  if (!N || !x || !target || nx < 1 || ny < 1 || nz < 1) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = ensure_workspace(N, nx, ny, nz);
  if (s != DTT_OK) return s;
  if ((s = upload_input(N, x)) != DTT_OK) return s;
  NCK(cudaMemcpyAsync(N->tgt, target, (size_t)N->d0.V() * 3 * sizeof(float), cudaMemcpyHostToDevice, N->stream));
  if ((s = forward(N)) != DTT_OK) return s;
  double l = 0.0;
  if ((s = backward(N, &l)) != DTT_OK) return s;
  if (loss) *loss = l;
  if (grad) {
    NCK(cudaMemcpyAsync(grad, N->g, N->np * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
    NCK(cudaStreamSynchronize(N->stream));
  }
  return DTT_OK;
}

dtt_status dtt_net_layer_trace(dtt_net* N, int32_t nx, int32_t ny, int32_t nz, const float* x, const float* target,
                               int32_t layer, float* act_in, float* dz, float* grad_w, float* grad_b,
                               float* grad_in) {
  if (!N || !x || !target || nx < 1 || ny < 1 || nz < 1 || layer < 0 || layer >= NLAYER)
    return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = ensure_workspace(N, nx, ny, nz);
  if (s != DTT_OK) return s;
  // the layer's level: full resolution (0, 1, 8, 9, 10), half (2, 3, 6, 7), quarter (4, 5)
  const Dims& d = (layer == 4 || layer == 5) ? N->d2 : ((layer >= 2 && layer <= 7) ? N->d1 : N->d0);
  const Layer& L = N->L[layer];
  const size_t nin = (size_t)d.V() * L.cin, nout = (size_t)d.V() * L.cout;
  if ((s = nalloc(&N->tr_in, nin * sizeof(bf16))) != DTT_OK) return s;
  if ((s = nalloc(&N->tr_dz, nout * sizeof(bf16))) != DTT_OK || (s = nalloc(&N->tr_dx, nin * sizeof(float))) != DTT_OK) {
    nfree(N->tr_in);
    nfree(N->tr_dz);
    return s;
  }
  cudaMemsetAsync(N->tr_dx, 0, nin * sizeof(float), N->stream);
  N->trace_layer = layer;
  s = upload_input(N, x);
  if (s == DTT_OK) {
    cudaError_t e = cudaMemcpyAsync(N->tgt, target, (size_t)N->d0.V() * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                    N->stream);
    if (e != cudaSuccess) s = set_error(DTT_ERR_CUDA, cudaGetErrorString(e));
  }
  if (s == DTT_OK) s = forward(N);
  if (s == DTT_OK) s = backward(N, nullptr);
  N->trace_layer = -1;
  std::vector<uint16_t> hin(nin), hdz(nout);
  if (s == DTT_OK) {
    cudaError_t e = cudaMemcpyAsync(hin.data(), N->tr_in, nin * sizeof(bf16), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hdz.data(), N->tr_dz, nout * sizeof(bf16), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess && grad_w)
      e = cudaMemcpyAsync(grad_w, N->g + L.woff, (size_t)27 * L.cin * L.cout * sizeof(float), cudaMemcpyDeviceToHost,
                          N->stream);
    if (e == cudaSuccess && grad_b)
      e = cudaMemcpyAsync(grad_b, N->g + L.boff, (size_t)L.cout * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess && grad_in)
      e = cudaMemcpyAsync(grad_in, N->tr_dx, nin * sizeof(float), cudaMemcpyDeviceToHost, N->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(N->stream);
    if (e != cudaSuccess) s = set_error(DTT_ERR_CUDA, cudaGetErrorString(e));
  }
  nfree(N->tr_in);
  nfree(N->tr_dz);
  nfree(N->tr_dx);
  if (s != DTT_OK) return s;
  // BF16 is the upper half of an FP32 word
  auto widen = [](uint16_t h) {
    const uint32_t w = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &w, sizeof(f));
    return f;
  };
  if (act_in)
    for (size_t q = 0; q < nin; ++q) act_in[q] = widen(hin[q]);
  if (dz)
    for (size_t q = 0; q < nout; ++q) dz[q] = widen(hdz[q]);
  return DTT_OK;
}

dtt_status dtt_net_forward(dtt_net* N, int32_t nx, int32_t ny, int32_t nz, const float* x, float* out) {
  if (!N || !x || !out || nx < 1 || ny < 1 || nz < 1) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = ensure_workspace(N, nx, ny, nz);
  if (s != DTT_OK) return s;
  if ((s = upload_input(N, x)) != DTT_OK) return s;
  if ((s = forward(N)) != DTT_OK) return s;
  const long long V = N->d0.V();
  std::vector<float> y((size_t)V * NET_COUT);
  NCK(cudaMemcpyAsync(y.data(), N->y, y.size() * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  for (long long v = 0; v < V; ++v)
    for (int c = 0; c < 3; ++c) out[v * 3 + c] = y[v * NET_COUT + c];
  return DTT_OK;
}

dtt_status dtt_net_features(dtt_net* N, dtt_grid* G, float* x) {
  if (!N || !G || !x) return set_error(DTT_ERR_ARG, "null argument");
  dtt_status s = grid_features(N, G, whole_grid(G));
  if (s != DTT_OK) return s;
  NCK(cudaMemcpyAsync(x, N->xf, (size_t)N->d0.V() * 16 * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  return DTT_OK;
}

dtt_status dtt_net_train_step(dtt_net* N, dtt_grid* G, const double* u_target, float lr, double* loss) {
  if (!N || !G || !u_target || !(lr > 0.f)) return set_error(DTT_ERR_ARG, "bad argument");
  double l = 0.0;
  dtt_status s = cell_loss_grad(N, G, u_target, &l);
  if (s != DTT_OK) return s;
  N->step += 1;
  NCKL(launch_adam(N->p, N->g, N->m, N->v, N->np, lr, N->step, N->stream));
  if ((s = refresh_bf16(N)) != DTT_OK) return s;
  NCK(cudaStreamSynchronize(N->stream));
  if (loss) *loss = l;
  return DTT_OK;
}

dtt_status dtt_net_grad_step(dtt_net* N, dtt_grid* G, const double* u_target, float* grad, double* loss) {
  if (!N || !G || !u_target || !grad) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = check_device_floats(grad, N->np, "grad");
  if (s != DTT_OK) return s;
  double l = 0.0;
  if ((s = cell_loss_grad(N, G, u_target, &l)) != DTT_OK) return s;
  NCK(cudaMemcpyAsync(grad, N->g, (size_t)N->np * sizeof(float), cudaMemcpyDeviceToDevice, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  if (loss) *loss = l;
  return DTT_OK;
}

dtt_status dtt_net_set_increment(dtt_net* N, float pressure_weight, float active_threshold, int32_t window_lateral,
                                 int32_t window_depth) {
  if (!N || !(pressure_weight >= 0.f) || !std::isfinite(active_threshold) || window_lateral < 0 || window_depth < 0)
    return set_error(DTT_ERR_ARG, "pressure_weight >= 0, a finite threshold and window sizes >= 0 required");
  N->inc_wp = pressure_weight;
  N->inc_thr = active_threshold;
  N->win_lat = window_lateral;
  N->win_dep = window_depth;
  return DTT_OK;
}

}  // extern "C"

namespace {
// surface nodes inside the window (the pressure term's count)
long long window_surface(const dtt_grid* G, const IncArgs& a) {
  long long n = 1;
  for (int d = 0; d < 3; ++d)
    if (d != G->c_axis) n *= a.w.n[d];
  return n;
}

// Features, targets, forward pass, loss and backward pass of increment k: the gradient in
// N->g and the loss in N->d_loss (on the net's stream, not synchronised).
dtt_status inc_loss_grad(dtt_net* N, dtt_grid* G, const double* u_prev2, const double* fn_prev,
                         const double depth[3], const double* u_target, const double* fn_target) {
  IncArgs a;
  dtt_status s = inc_setup(N, G, u_prev2, fn_prev, depth, a);
  if (s != DTT_OK) return s;
  cudaStream_t st = N->stream;
  NCKL(launch_inc_targets(a, u_target, fn_target, N->inc_t, N->inc_m, st));
  if ((s = forward(N)) != DTT_OK) return s;
  NCK(cudaMemsetAsync(N->g, 0, (size_t)N->np * sizeof(float), st));
  NCK(cudaMemsetAsync(N->d_loss, 0, sizeof(double), st));
  const float wp = N->inc_wp / (float)window_surface(G, a);
  NCKL(launch_inc_loss(N->y, N->inc_t, N->inc_m, N->d0.V(), NET_COUT, wp, N->gP, N->d_loss, st));
  return bwd_chain(N);
}

// DTT_ERR_ARG unless p points into managed memory or device memory of the current device
// (the net's): a kernel given a plain host pointer, or another GPU's memory without peer
// access, would fault
dtt_status check_device_floats(const float* p, long long n, const char* what) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DTT_ERR_ARG, std::string(what) + ": not a CUDA pointer");
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return set_error(DTT_ERR_ARG, std::string(what) + ": device memory of " + std::to_string(n) + " floats required");
  int cur = -1;
  NCK(cudaGetDevice(&cur));
  if (at.type == cudaMemoryTypeDevice && at.device != cur)
    return set_error(DTT_ERR_ARG, std::string(what) + ": memory of device " + std::to_string(at.device) +
                                      ", not of the current device " + std::to_string(cur));
  return DTT_OK;
}
}  // namespace

extern "C" {

dtt_status dtt_net_increment_features(dtt_net* N, dtt_grid* G, const double* u_prev2, const double* fn_prev,
                                      const double depth[3], float* x) {
  if (!N || !G) return set_error(DTT_ERR_ARG, "null argument");
  IncArgs a;
  dtt_status s = inc_setup(N, G, u_prev2, fn_prev, depth, a);
  if (s != DTT_OK) return s;
  if (x) NCK(cudaMemcpyAsync(x, N->xf, (size_t)N->d0.V() * 16 * sizeof(float), cudaMemcpyDeviceToHost, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  return DTT_OK;
}

dtt_status dtt_net_train_increment(dtt_net* N, dtt_grid* G, const double* u_prev2, const double* fn_prev,
                                   const double depth[3], const double* u_target, const double* fn_target, float lr,
                                   double* loss) {
  if (!N || !G || !u_target || !fn_target || !(lr > 0.f)) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = inc_loss_grad(N, G, u_prev2, fn_prev, depth, u_target, fn_target);
  if (s != DTT_OK) return s;
  cudaStream_t st = N->stream;
  double l = 0.0;
  NCK(cudaMemcpyAsync(&l, N->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  N->step += 1;
  NCKL(launch_adam(N->p, N->g, N->m, N->v, N->np, lr, N->step, st));
  if ((s = refresh_bf16(N)) != DTT_OK) return s;
  NCK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return DTT_OK;
}

dtt_status dtt_net_grad_increment(dtt_net* N, dtt_grid* G, const double* u_prev2, const double* fn_prev,
                                  const double depth[3], const double* u_target, const double* fn_target, float* grad,
                                  double* loss) {
  if (!N || !G || !u_target || !fn_target || !grad) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = check_device_floats(grad, N->np, "grad");
  if (s != DTT_OK) return s;
  if ((s = inc_loss_grad(N, G, u_prev2, fn_prev, depth, u_target, fn_target)) != DTT_OK) return s;
  cudaStream_t st = N->stream;
  double l = 0.0;
  NCK(cudaMemcpyAsync(&l, N->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  NCK(cudaMemcpyAsync(grad, N->g, (size_t)N->np * sizeof(float), cudaMemcpyDeviceToDevice, st));
  NCK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return DTT_OK;
}

dtt_status dtt_net_apply_grad(dtt_net* N, const float* grad, float scale, float lr) {
  if (!N || !grad || !(lr > 0.f) || !(scale > 0.f) || !std::isfinite(scale))
    return set_error(DTT_ERR_ARG, "a gradient, lr > 0 and a finite scale > 0 required");
  dtt_status s = check_device_floats(grad, N->np, "grad");
  if (s != DTT_OK) return s;
  cudaStream_t st = N->stream;
  N->step += 1;
  NCKL(launch_adam(N->p, grad, N->m, N->v, N->np, lr, N->step, st, scale));
  if ((s = refresh_bf16(N)) != DTT_OK) return s;
  NCK(cudaStreamSynchronize(st));
  return DTT_OK;
}

dtt_status dtt_net_predict_increment(dtt_net* N, dtt_grid* G, const double* u_prev2, const double* fn_prev,
                                     const double depth[3]) {
  if (!N || !G) return set_error(DTT_ERR_ARG, "null argument");
  IncArgs a;
  dtt_status s = inc_setup(N, G, u_prev2, fn_prev, depth, a);
  if (s != DTT_OK) return s;
  if (N->act_cap < G->nface) {
    nfree(N->d_act);
    N->act_cap = 0;
    if ((s = nalloc(&N->d_act, (size_t)G->nface)) != DTT_OK) return s;
    N->act_cap = G->nface;
  }
  if (N->ug_cap < 3 * G->NN) {
    nfree(N->d_ug);
    N->ug_cap = 0;
    if ((s = nalloc(&N->d_ug, (size_t)(3 * G->NN) * sizeof(double))) != DTT_OK) return s;
    N->ug_cap = 3 * G->NN;
  }
  if ((s = forward(N)) != DTT_OK) return s;
  NCKL(launch_inc_guess(a, N->y, NET_COUT, N->inc_thr, N->d_ug, N->d_act, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  return set_guess_with_fallback(G, N->d_ug, N->d_act);
}

dtt_status dtt_net_loss_grad_increment(dtt_net* N, int32_t nx, int32_t ny, int32_t nz, const float* x,
                                       const float* target, const float* pmask, double* loss, float* grad) {
  if (!N || !x || !target || !pmask || nx < 1 || ny < 1 || nz < 1) return set_error(DTT_ERR_ARG, "bad argument");
  dtt_status s = ensure_workspace(N, nx, ny, nz);
  if (s != DTT_OK) return s;
  if ((s = upload_input(N, x)) != DTT_OK) return s;
  const long long V = N->d0.V();
  cudaStream_t st = N->stream;
  NCK(cudaMemcpyAsync(N->inc_t, target, (size_t)V * 4 * sizeof(float), cudaMemcpyHostToDevice, st));
  NCK(cudaMemcpyAsync(N->inc_m, pmask, (size_t)V * sizeof(float), cudaMemcpyHostToDevice, st));
  double ns = 0.0;
  for (long long v = 0; v < V; ++v) ns += pmask[v] != 0.f ? 1.0 : 0.0;
  if ((s = forward(N)) != DTT_OK) return s;
  NCK(cudaMemsetAsync(N->g, 0, (size_t)N->np * sizeof(float), st));
  NCK(cudaMemsetAsync(N->d_loss, 0, sizeof(double), st));
  const float wp = ns > 0.0 ? N->inc_wp / (float)ns : 0.f;
  NCKL(launch_inc_loss(N->y, N->inc_t, N->inc_m, V, NET_COUT, wp, N->gP, N->d_loss, st));
  if ((s = bwd_chain(N)) != DTT_OK) return s;
  double l = 0.0;
  NCK(cudaMemcpyAsync(&l, N->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (grad) NCK(cudaMemcpyAsync(grad, N->g, N->np * sizeof(float), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return DTT_OK;
}

dtt_status dtt_net_predict(dtt_net* N, dtt_grid* G) {
  if (!N || !G) return set_error(DTT_ERR_ARG, "null argument");
  dtt_status s = grid_features(N, G, whole_grid(G));
  if (s != DTT_OK) return s;
  if ((s = forward(N)) != DTT_OK) return s;
  NCKL(launch_out_to_u(N->y, N->d0.V(), NET_COUT, u_scale(G), N->d_u, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  return dtt_set_initial(G, N->d_u, 1);
}

}  // extern "C"

// Constraint projections, contact evaluation, Anderson acceleration and the device-side
// control of the fixed-point iteration.
//
//  * proj_P (Eq. 9, 14, 17): lambda_r = (sum_e a_e p_e) / (sum_e a_e b_e), p_e -= b_e lambda_r,
//    multiplier f_r = -lambda_r kept in FP64.  The same shift is applied to p~ (= p + A0 u~).
//  * proj_U (Eq. 9, 11, 15): u~_e += a_e (t_r - sum a u~) / (sum a a), in FP64.
//  * Contact (Section 5.1, Eq. 24-28, Algorithm 2): gap g = |O - M'| - R, normal
//    n_c = (O - M')/|O - M'| with M' = M + u* + u~ (FP64); on the active set C,
//    p <- p - (p.n_c) n_c; normal reaction f = -h^3 sum_c W_c p_c n_c (one-sided divergence,
//    evaluated before the projection); violation sets V_gap = {M not in C: g < 0},
//    V_react = {M in C: f > 0}; proj_U places an active node radially on the sphere,
//    u(M) = O - R n_c - M.
//  * Anderson depth 4 (Section 4.1.1): R_{i-1} = x_i - S_{i-1}; every mod_ACV iterations
//    after the first four, alpha = argmin ||sum alpha_k R_k|| with sum alpha_k = 1 (FP64
//    Gram, Gaussian elimination with partial pivoting, skipped on a pivot <= acv_pivot max G_kk),
//    x_i <- sum alpha_k (S_k + R_k).
// All scalar decisions run in single-thread control kernels so that an iteration is a fixed
// sequence of launches; every kernel returns at once when the solve is finished.
#include <cstddef>

#include "dtt_internal.cuh"

namespace dtt {

constexpr int SB = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  #pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;   // valid in thread 0
}

__device__ __forceinline__ double read_u(long long e, const double* u64, const float* uhi, const float* ulo) {
  return u64 ? u64[e] : (double)uhi[e] + (double)ulo[e];
}
__device__ __forceinline__ void write_u(long long e, double v, double* u64, float* uhi, float* ulo) {
  if (u64) u64[e] = v;
  else { float h, l; ff_set(h, l, v); uhi[e] = h; ulo[e] = l; }
}

__device__ __forceinline__ void node_ijk(const GridDev& g, long long n, int& i, int& j, int& k) {
  i = (int)(n % g.nn[0]);
  long long r = n / g.nn[0];
  j = (int)(r % g.nn[1]);
  k = (int)(r / g.nn[1]);
}

__device__ __forceinline__ void node_W(const GridDev& g, int c, int i, int j, int k, bool& dof, double& W) {
  W = 1.0;
  dof = true;
  const int idx[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) {
    if (g.periodic[d]) continue;
    int f = -1;
    if (idx[d] == 0) f = 0;
    else if (idx[d] == g.nn[d] - 1) f = 1;
    if (f < 0) continue;
    int t = g.bc[d][f][c];
    if (t == BC_D) dof = false;
    else if (t == BC_N) W *= 0.5;
  }
}

// ------------------------------------------------------------------ proj_P (rows)
template <typename T>
__device__ __forceinline__ void pick_p(const Ctrl* ctrl, int ring_mode, T* p_direct, void* const* pring,
                                       void* const* rring, T*& p, T*& shadow) {
  p = p_direct;
  shadow = nullptr;
  if (ring_mode) {
    const int il = ctrl->i_local;
    p = (T*)pring[il % 4];
    if (il > 0) shadow = (T*)rring[(il - 1) % 4];
  }
}

// Gram-row contributions <R_new, R_k> of one DOF (fused Gram mode).
template <typename T>
__device__ __forceinline__ void gram_add(double* G, void* const* rring, int rslot, long long d) {
  const double rn = (double)((const T*)rring[rslot])[d];
  #pragma unroll
  for (int q = 0; q < 4; ++q) G[q] += rn * (q == rslot ? rn : (double)((const T*)rring[q])[d]);
}

template <typename T>
__global__ void k_proj_P(const RowsDev r, T* p_direct, void* const* pring, void* const* rring, int ring_mode,
                         int gram, double* partials, const Ctrl* ctrl, T* step_clear) {
  __shared__ double sh[SB / 32];
  if (ctrl && ctrl->done) return;
  T *p, *x;
  pick_p<T>(ctrl, ring_mode, p_direct, pring, rring, p, x);
  const int rslot = (ring_mode && ctrl->i_local > 0) ? (ctrl->i_local - 1) % 4 : -1;
  double acc = 0.0;
  double G[4] = {0, 0, 0, 0};
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row < r.nrows) {
    double sap = 0.0;
    for (int e = r.ptr[row]; e < r.ptr[row + 1]; ++e) sap += r.a[e] * (double)p[r.dof[e]];
    double lam = sap / r.ab[row];
    for (int e = r.ptr[row]; e < r.ptr[row + 1]; ++e) {
      long long d = r.dof[e];
      double sh_ = r.b[e] * lam;
      double pn = (double)p[d] - sh_;
      p[d] = (T)pn;
      if (x) x[d] = (T)((double)x[d] - sh_);
      acc += (double)(T)pn * (double)(T)pn;
      if (gram && rslot >= 0) gram_add<T>(G, rring, rslot, d);
      // exact residual mode: the residual kernel has read this iteration's step; the
      // row's DOFs start the next correction from zero
      if (step_clear) step_clear[d] = (T)0;
    }
    r.mult[row] = -lam;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[PROJ_STRIDE * blockIdx.x] = t;
  for (int q = 0; q < 4; ++q) {
    double tq = block_sum(G[q], sh);
    if (threadIdx.x == 0) partials[PROJ_STRIDE * blockIdx.x + 1 + q] = tq;
  }
}

template <typename T>
int launch_proj_P_rows(const GridDev& g, const RowsDev& r, T* p_direct, void* const* pring, void* const* rring,
                       int ring_mode, int gram, double* partials, const Ctrl* ctrl, cudaStream_t s, T* step_clear) {
  (void)g;
  int blocks = (r.nrows + SB - 1) / SB;
  if (blocks == 0) return 0;
  k_proj_P<T><<<blocks, SB, 0, s>>>(r, p_direct, pring, rring, ring_mode, gram, partials, ctrl, step_clear);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ proj_U (rows)
// The correction applied to u~ is also added to the step field (the Anderson difference
// form needs the full step u~_{i+1} - u~_i).
// end: when set, the CTA that finishes last advances the iteration counters (k_ctrl_end).
template <typename T>
__global__ void k_proj_U(const RowsDev r, double* u64, float* uhi, float* ulo, T* step, const Ctrl* ctrl,
                         Ctrl* end) {
  if (ctrl && ctrl->done) return;
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row < r.nrows) {
    double sau = 0.0;
    for (int e = r.ptr[row]; e < r.ptr[row + 1]; ++e) sau += r.a[e] * read_u(r.dof[e], u64, uhi, ulo);
    double corr = (r.target[row] - sau) / r.aa[row];
    for (int e = r.ptr[row]; e < r.ptr[row + 1]; ++e) {
      if (r.a[e] == 0.0) continue;
      long long d = r.dof[e];
      double du = r.a[e] * corr;
      write_u(d, read_u(d, u64, uhi, ulo) + du, u64, uhi, ulo);
      if (step) step[d] = (T)((double)step[d] + du);
    }
  }
  if (end && threadIdx.x == 0) {
    // every CTA passed the done test above before its count; the last one to count ends
    // the iteration and clears the count for the next
    if (atomicAdd(&end->blocks_done, 1u) == gridDim.x - 1) {
      end->iter += 1;
      end->i_local += 1;
      end->blocks_done = 0;
    }
  }
}

template <typename T>
int launch_proj_U_rows(const GridDev& g, const RowsDev& r, double* u64, float* uhi, float* ulo, T* step,
                       const Ctrl* ctrl, cudaStream_t s) {
  (void)g;
  int blocks = (r.nrows + SB - 1) / SB;
  if (blocks == 0) return 0;
  k_proj_U<T><<<blocks, SB, 0, s>>>(r, u64, uhi, ulo, step, ctrl, nullptr);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_proj_U_rows_end(const GridDev& g, const RowsDev& r, double* u64, float* uhi, float* ulo, T* step,
                           Ctrl* ctrl, cudaStream_t s) {
  (void)g;
  int blocks = (r.nrows + SB - 1) / SB;
  if (blocks == 0) return launch_ctrl_end(ctrl, s);
  k_proj_U<T><<<blocks, SB, 0, s>>>(r, u64, uhi, ulo, step, ctrl, ctrl);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ contact
int contact_blocks(int nface) { return (nface + SB - 1) / SB; }

__device__ void contact_geom(const ContactArgs& a, long long n, double Mp[3], double nv[3], double& gap,
                             double X[3]) {
  int i, j, k;
  node_ijk(a.g, n, i, j, k);
  X[0] = a.g.h * i; X[1] = a.g.h * j; X[2] = a.g.h * k;
  double v[3], dist2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    double us = a.eps[c][0] * X[0] + a.eps[c][1] * X[1] + a.eps[c][2] * X[2];
    Mp[c] = X[c] + us + read_u((long long)c * a.g.nnodes + n, a.u64, a.uhi, a.ulo);
    v[c] = a.c.center[c] - Mp[c];
    dist2 += v[c] * v[c];
  }
  double dist = sqrt(dist2);
  for (int c = 0; c < 3; ++c) nv[c] = v[c] / dist;
  gap = dist - a.c.radius;
}

template <typename T>
__global__ void k_contact_eval(const ContactArgs a, T* p_direct, void* const* pring, void* const* rring,
                               int ring_mode, int gram) {
  __shared__ double sh[SB / 32];
  if (a.ctrl && a.ctrl->done) return;
  T *p, *x;
  pick_p<T>(a.ctrl, ring_mode, p_direct, pring, rring, p, x);
  const int rslot = (ring_mode && a.ctrl->i_local > 0) ? (a.ctrl->i_local - 1) % 4 : -1;
  double G[4] = {0, 0, 0, 0};
  double p2 = 0.0, ng = 0.0, nr = 0.0, mm = 0.0;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < a.c.nnodes_face) {
    long long n = a.c.node[q];
    double Mp[3], nv[3], X[3], gap;
    contact_geom(a, n, Mp, nv, gap, X);
    int i, j, k;
    node_ijk(a.g, n, i, j, k);
    double pv[3], W[3];
    bool dof[3];
    double f = 0.0, pn = 0.0;
    for (int c = 0; c < 3; ++c) {
      node_W(a.g, c, i, j, k, dof[c], W[c]);
      pv[c] = dof[c] ? (double)p[(long long)c * a.g.nnodes + n] : 0.0;
      f += W[c] * pv[c] * nv[c];
      pn += pv[c] * nv[c];
    }
    f *= -(a.g.h * a.g.h * a.g.h);
    const bool act = a.c.active[q] != 0;
    if (act) {
      for (int c = 0; c < 3; ++c) {
        if (!dof[c]) continue;
        long long e = (long long)c * a.g.nnodes + n;
        double sh_ = pn * nv[c];
        double np_ = pv[c] - sh_;
        p[e] = (T)np_;
        if (x) x[e] = (T)((double)x[e] - sh_);
        pv[c] = (double)(T)np_;
      }
    }
    for (int c = 0; c < 3; ++c) p2 += pv[c] * pv[c];
    if (gram && rslot >= 0)
      for (int c = 0; c < 3; ++c)
        if (dof[c]) gram_add<T>(G, rring, rslot, (long long)c * a.g.nnodes + n);
    uint8_t vg = (!act && gap < 0.0) ? 1 : 0;
    uint8_t vr = (act && f > 0.0) ? 1 : 0;
    if (vg != a.c.vgap_prev[q] || vr != a.c.vreact_prev[q]) mm = 1.0;
    a.c.vgap[q] = vg;
    a.c.vreact[q] = vr;
    ng = vg;
    nr = vr;
    a.c.gap[q] = gap;
    a.c.fn[q] = f;
    for (int c = 0; c < 3; ++c) a.c.nvec[3 * q + c] = nv[c];
    // exact residual mode: the residual kernel has read this iteration's step; the face
    // nodes start the next correction from zero
    if (a.step_clear)
      for (int c = 0; c < 3; ++c) ((T*)a.step_clear)[(long long)c * a.g.nnodes + n] = (T)0;
  }
  double t0 = block_sum(p2, sh);
  double t1 = block_sum(ng, sh);
  double t2 = block_sum(nr, sh);
  double t3 = block_sum(mm, sh);
  if (threadIdx.x == 0) {
    a.partials[CONT_STRIDE * blockIdx.x] = t0;
    a.partials[CONT_STRIDE * blockIdx.x + 1] = t1;
    a.partials[CONT_STRIDE * blockIdx.x + 2] = t2;
    a.partials[CONT_STRIDE * blockIdx.x + 3] = t3;
  }
  for (int q = 0; q < 4; ++q) {
    double tq = block_sum(G[q], sh);
    if (threadIdx.x == 0) a.partials[CONT_STRIDE * blockIdx.x + 4 + q] = tq;
  }
}

template <typename T>
int launch_contact_eval(const ContactArgs& a, T* p_direct, void* const* pring, void* const* rring, int ring_mode,
                        int gram, cudaStream_t s) {
  int blocks = contact_blocks(a.c.nnodes_face);
  if (blocks == 0) return 0;
  k_contact_eval<T><<<blocks, SB, 0, s>>>(a, p_direct, pring, rring, ring_mode, gram);
  return (int)cudaGetLastError();
}

__global__ void k_contact_update(const ContactArgs a) {
  Ctrl* ctrl = const_cast<Ctrl*>(a.ctrl);
  if (ctrl->done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.c.nnodes_face) return;
  uint8_t vg = a.c.vgap[q], vr = a.c.vreact[q];
  if (ctrl->update) {
    uint8_t old = a.c.active[q];
    uint8_t nw = (uint8_t)((old | vg) & (vr ? 0 : 1));
    if (nw != old) { a.c.active[q] = nw; atomicAdd(&ctrl->changed, 1); }
  }
  a.c.vgap_prev[q] = vg;
  a.c.vreact_prev[q] = vr;
}

int launch_contact_update(const ContactArgs& a, cudaStream_t s) {
  int blocks = contact_blocks(a.c.nnodes_face);
  if (blocks == 0) return 0;
  k_contact_update<<<blocks, SB, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <typename T>
__global__ void k_contact_proj_U(const ContactArgs a, double* u64, float* uhi, float* ulo, T* step) {
  if (a.ctrl && a.ctrl->done) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.c.nnodes_face || !a.c.active[q]) return;
  long long n = a.c.node[q];
  double Mp[3], nv[3], X[3], gap;
  contact_geom(a, n, Mp, nv, gap, X);
  int i, j, k;
  node_ijk(a.g, n, i, j, k);
  for (int c = 0; c < 3; ++c) {
    bool dof;
    double W;
    node_W(a.g, c, i, j, k, dof, W);
    if (!dof) continue;
    double us = a.eps[c][0] * X[0] + a.eps[c][1] * X[1] + a.eps[c][2] * X[2];
    double target = a.c.center[c] - a.c.radius * nv[c] - X[c] - us;
    const long long e = (long long)c * a.g.nnodes + n;
    if (step) step[e] = (T)((double)step[e] + (target - read_u(e, u64, uhi, ulo)));
    write_u(e, target, u64, uhi, ulo);
  }
}

template <typename T>
int launch_contact_proj_U(const ContactArgs& a, double* u64, float* uhi, float* ulo, T* step, cudaStream_t s) {
  int blocks = contact_blocks(a.c.nnodes_face);
  if (blocks == 0) return 0;
  k_contact_proj_U<T><<<blocks, SB, 0, s>>>(a, u64, uhi, ulo, step);
  return (int)cudaGetLastError();
}

// Initial contact zone of an increment: C = {g < 0} at the starting field (Section 5.1.3),
// or, with keep_active, the zone the caller set (dtt_set_initial_contact).
__global__ void k_contact_init(const ContactArgs a, int keep_active) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.c.nnodes_face) return;
  long long n = a.c.node[q];
  double Mp[3], nv[3], X[3], gap;
  contact_geom(a, n, Mp, nv, gap, X);
  if (!keep_active) a.c.active[q] = gap < 0.0 ? 1 : 0;
  a.c.vgap_prev[q] = 0;
  a.c.vreact_prev[q] = 0;
  a.c.gap[q] = gap;
}

int launch_contact_init(const ContactArgs& a, cudaStream_t s, int keep_active) {
  int blocks = contact_blocks(a.c.nnodes_face);
  if (blocks == 0) return 0;
  k_contact_init<<<blocks, SB, 0, s>>>(a, keep_active);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ Anderson
int acv_blocks(const GridDev& g) {
  long long total = 3 * g.nnodes;
  return (int)std::min<long long>((total + SB - 1) / SB, 148LL * 8);
}

// storeR: R_{i-1} = x_i - S_{i-1}, and its dot products with the four ring slots.
template <typename T>
__global__ void k_acv_store(long long total, int acv_on, void* const* S, void* const* R, const double* u64,
                            double* partials, const Ctrl* ctrl) {
  __shared__ double sh[SB / 32];
  if (ctrl->done) return;
  const int i = ctrl->i_local;
  if (i <= 0) return;
  const T* x = (acv_on == 1) ? (const T*)S[i % 5] : nullptr;
  const T* sp = (const T*)S[(i - 1) % 5];
  const int rs = (i - 1) % 4;
  T* Rn = (T*)R[rs];
  const T* R0 = (const T*)R[0];
  const T* R1 = (const T*)R[1];
  const T* R2 = (const T*)R[2];
  const T* R3 = (const T*)R[3];
  double d[4] = {0, 0, 0, 0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    T xv = (acv_on == 1) ? x[e] : (T)u64[e];
    T rv = xv - sp[e];
    Rn[e] = rv;
    double r = (double)rv;
    d[0] += r * (double)(rs == 0 ? rv : R0[e]);
    d[1] += r * (double)(rs == 1 ? rv : R1[e]);
    d[2] += r * (double)(rs == 2 ? rv : R2[e]);
    d[3] += r * (double)(rs == 3 ? rv : R3[e]);
  }
  for (int k = 0; k < 4; ++k) {
    double t = block_sum(d[k], sh);
    if (threadIdx.x == 0) partials[4 * blockIdx.x + k] = t;
  }
}

template <typename T>
int launch_acv_store(const GridDev& g, int acv_on, void* const* Sring, void* const* Rring,
                     const double* u64, double* partials, const Ctrl* ctrl, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  k_acv_store<T><<<acv_blocks(g), SB, 0, s>>>(total, acv_on, Sring, Rring, u64, partials, ctrl);
  return (int)cudaGetLastError();
}

// Gram row of the newest Anderson residual R_{i-1} (difference form).
template <typename T>
__global__ void k_acv_gram(long long total, void* const* R, double* partials, const Ctrl* ctrl) {
  __shared__ double sh[SB / 32];
  if (ctrl->done) return;
  const int i = ctrl->i_local;
  if (i <= 0) return;
  const int rs = (i - 1) % 4;
  const T* Rn = (const T*)R[rs];
  const T* R0 = (const T*)R[0];
  const T* R1 = (const T*)R[1];
  const T* R2 = (const T*)R[2];
  const T* R3 = (const T*)R[3];
  T d0 = 0, d1 = 0, d2 = 0, d3 = 0;   // per-thread partial sums in T; block and grid sums in FP64
  double D[4] = {0, 0, 0, 0};
  int cnt = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const T r = Rn[e];
    d0 += r * R0[e];
    d1 += r * R1[e];
    d2 += r * R2[e];
    d3 += r * R3[e];
    if (++cnt == 16) {
      D[0] += (double)d0; D[1] += (double)d1; D[2] += (double)d2; D[3] += (double)d3;
      d0 = d1 = d2 = d3 = 0;
      cnt = 0;
    }
  }
  D[0] += (double)d0; D[1] += (double)d1; D[2] += (double)d2; D[3] += (double)d3;
  for (int k = 0; k < 4; ++k) {
    double t = block_sum(D[k], sh);
    if (threadIdx.x == 0) partials[4 * blockIdx.x + k] = t;
  }
}

template <typename T>
int launch_acv_gram(const GridDev& g, void* const* rring, double* partials, const Ctrl* ctrl, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  k_acv_gram<T><<<acv_blocks(g), SB, 0, s>>>(total, rring, partials, ctrl);
  return (int)cudaGetLastError();
}

// Green input of iteration i: p_i, or the Anderson combination in difference form
//   g_i = sum_m alpha_m p_{i-3+m} - sum_{q=0..2} beta_q (R_{i-3+q} - p_{i-2+q} + g_{i-3+q}),
//   beta_q = alpha_0 + ... + alpha_q.
// (x_{j+1} = p_{j+1} + A0 u~_{j+1}, S_j = A0 u~_j + g_j, R_j = x_{j+1} - S_j, hence
//  sum alpha_j x_{j+1} - A0 u~_i = sum alpha_j p_{j+1} - sum_k beta_k A0 Delta_k with
//  A0 Delta_k = R_k - p_{k+1} + g_k.)
template <typename T>
__global__ void k_acv_green_input(long long total, void* const* P, void* const* Gr, void* const* R,
                                  const Ctrl* ctrl) {
  if (ctrl->done) return;
  const int i = ctrl->i_local;
  T* gi = (T*)Gr[i % 4];
  if (!ctrl->accel) {
    const T* pi = (const T*)P[ctrl->i_local == 0 ? ctrl->pslot : i % 4];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
      gi[e] = pi[e];
    return;
  }
  const T a0 = (T)ctrl->alpha[0], a1 = (T)ctrl->alpha[1], a2 = (T)ctrl->alpha[2], a3 = (T)ctrl->alpha[3];
  const T b0 = a0, b1 = a0 + a1, b2 = a0 + a1 + a2;
  const T* p0 = (const T*)P[(i - 3) % 4];
  const T* p1 = (const T*)P[(i - 2) % 4];
  const T* p2 = (const T*)P[(i - 1) % 4];
  const T* p3 = (const T*)P[i % 4];
  const T* r0 = (const T*)R[(i - 3) % 4];
  const T* r1 = (const T*)R[(i - 2) % 4];
  const T* r2 = (const T*)R[(i - 1) % 4];
  const T* g0 = (const T*)Gr[(i - 3) % 4];
  const T* g1 = (const T*)Gr[(i - 2) % 4];
  const T* g2 = (const T*)Gr[(i - 1) % 4];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const T q0 = p0[e], q1 = p1[e], q2 = p2[e], q3 = p3[e];
    T v = a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3;
    v -= b0 * (r0[e] - q1 + g0[e]);
    v -= b1 * (r1[e] - q2 + g1[e]);
    v -= b2 * (r2[e] - q3 + g2[e]);
    gi[e] = v;
  }
}

// FP32 form of k_acv_green_input on float4 vectors (ring fields are 256-byte aligned; the
// last total % 4 values take the scalar path), same arithmetic per value.
__device__ __forceinline__ float acv_combine(float q0, float q1, float q2, float q3, float r0, float r1, float r2,
                                             float g0, float g1, float g2, float a0, float a1, float a2, float a3,
                                             float b0, float b1, float b2) {
  float v = a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3;
  v -= b0 * (r0 - q1 + g0);
  v -= b1 * (r1 - q2 + g1);
  v -= b2 * (r2 - q3 + g2);
  return v;
}
// the same combination where R_k = p_(k+1) (exact residual mode away from constrained DOFs):
// R_k - p_(k+1) + g_k is then g_k exactly, so the result is the same bit for bit
__device__ __forceinline__ float acv_combine_free(float q0, float q1, float q2, float q3, float g0, float g1, float g2,
                                                  float a0, float a1, float a2, float a3, float b0, float b1, float b2) {
  float v = a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3;
  v -= b0 * g0;
  v -= b1 * g1;
  v -= b2 * g2;
  return v;
}

__global__ void k_acv_green_input_v4(long long total, void* const* P, void** Gr, void* const* Gown, void* const* R,
                                     const Ctrl* ctrl, int alias) {
  if (ctrl->done) return;
  const int i = ctrl->i_local;
  float* gi = (float*)Gown[i % 4];
  const long long n4 = total / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // one thread sets this iteration's ring entry; the blocks read only the other entries
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (!ctrl->accel) {
    const int src = i == 0 ? ctrl->pslot : i % 4;
    const float* pi = (const float*)P[src];
    // g_i = p_i: the ring entry can point at p_i itself when its slot is i % 4, since the
    // residual kernel rewrites that slot only at iteration i + 4, after g_i's last reader
    if (alias && src == i % 4) {
      if (lead) Gr[i % 4] = (void*)pi;
      return;
    }
    if (lead) Gr[i % 4] = gi;
    for (long long e = t0; e < n4; e += stride) ((float4*)gi)[e] = ((const float4*)pi)[e];
    for (long long e = 4 * n4 + t0; e < total; e += stride) gi[e] = pi[e];
    return;
  }
  if (lead) Gr[i % 4] = gi;
  // FP32 copies made by the control kernel: no per-thread FP64 conversion
  const float a0 = ctrl->alpha_f[0], a1 = ctrl->alpha_f[1], a2 = ctrl->alpha_f[2], a3 = ctrl->alpha_f[3];
  const float b0 = a0, b1 = a0 + a1, b2 = a0 + a1 + a2;
  const float* p0 = (const float*)P[(i - 3) % 4];
  const float* p1 = (const float*)P[(i - 2) % 4];
  const float* p2 = (const float*)P[(i - 1) % 4];
  const float* p3 = (const float*)P[i % 4];
  const float* r0 = (const float*)R[(i - 3) % 4];
  const float* r1 = (const float*)R[(i - 2) % 4];
  const float* r2 = (const float*)R[(i - 1) % 4];
  const float* g0 = (const float*)Gr[(i - 3) % 4];
  const float* g1 = (const float*)Gr[(i - 2) % 4];
  const float* g2 = (const float*)Gr[(i - 1) % 4];
  if (alias) {
    // exact residual mode: R_k = p_(k+1) bit for bit outside the tiles that hold constrained
    // DOFs (their flux and projections), so the R ring is not read here; k_acv_green_fix
    // recomputes those tiles' nodes from the full formula
    for (long long e = t0; e < n4; e += stride) {
      const float4 q0 = ((const float4*)p0)[e], q1 = ((const float4*)p1)[e], q2 = ((const float4*)p2)[e],
                   q3 = ((const float4*)p3)[e];
      const float4 h0 = ((const float4*)g0)[e], h1 = ((const float4*)g1)[e], h2 = ((const float4*)g2)[e];
      float4 v;
      v.x = acv_combine_free(q0.x, q1.x, q2.x, q3.x, h0.x, h1.x, h2.x, a0, a1, a2, a3, b0, b1, b2);
      v.y = acv_combine_free(q0.y, q1.y, q2.y, q3.y, h0.y, h1.y, h2.y, a0, a1, a2, a3, b0, b1, b2);
      v.z = acv_combine_free(q0.z, q1.z, q2.z, q3.z, h0.z, h1.z, h2.z, a0, a1, a2, a3, b0, b1, b2);
      v.w = acv_combine_free(q0.w, q1.w, q2.w, q3.w, h0.w, h1.w, h2.w, a0, a1, a2, a3, b0, b1, b2);
      ((float4*)gi)[e] = v;
    }
    for (long long e = 4 * n4 + t0; e < total; e += stride)
      gi[e] = acv_combine_free(p0[e], p1[e], p2[e], p3[e], g0[e], g1[e], g2[e], a0, a1, a2, a3, b0, b1, b2);
    return;
  }
  for (long long e = t0; e < n4; e += stride) {
    const float4 q0 = ((const float4*)p0)[e], q1 = ((const float4*)p1)[e], q2 = ((const float4*)p2)[e],
                 q3 = ((const float4*)p3)[e];
    const float4 s0 = ((const float4*)r0)[e], s1 = ((const float4*)r1)[e], s2 = ((const float4*)r2)[e];
    const float4 h0 = ((const float4*)g0)[e], h1 = ((const float4*)g1)[e], h2 = ((const float4*)g2)[e];
    float4 v;
    v.x = acv_combine(q0.x, q1.x, q2.x, q3.x, s0.x, s1.x, s2.x, h0.x, h1.x, h2.x, a0, a1, a2, a3, b0, b1, b2);
    v.y = acv_combine(q0.y, q1.y, q2.y, q3.y, s0.y, s1.y, s2.y, h0.y, h1.y, h2.y, a0, a1, a2, a3, b0, b1, b2);
    v.z = acv_combine(q0.z, q1.z, q2.z, q3.z, s0.z, s1.z, s2.z, h0.z, h1.z, h2.z, a0, a1, a2, a3, b0, b1, b2);
    v.w = acv_combine(q0.w, q1.w, q2.w, q3.w, s0.w, s1.w, s2.w, h0.w, h1.w, h2.w, a0, a1, a2, a3, b0, b1, b2);
    ((float4*)gi)[e] = v;
  }
  for (long long e = 4 * n4 + t0; e < total; e += stride)
    gi[e] = acv_combine(p0[e], p1[e], p2[e], p3[e], r0[e], r1[e], r2[e], g0[e], g1[e], g2[e], a0, a1, a2, a3, b0, b1,
                        b2);
}

// The accelerated Green input at the nodes of the tiles that hold constrained DOFs (one CTA
// per xy tile of the mixed residual kernel, tx x ty node columns, plus the final column in a
// wide last x tile, threads tx ty ..; its z range tile_z +- 1 layer): the full formula, after
// k_acv_green_input_v4 has written the R-free form everywhere.
__global__ void k_acv_green_fix(const GridDev g, void* const* P, void* const* Gr, void* const* Gown, void* const* R,
                                const Ctrl* ctrl, const int2* __restrict__ tile_z, int tx, int ty) {
  if (ctrl->done || !ctrl->accel) return;
  const int2 zr = tile_z[blockIdx.x];
  if (zr.x > zr.y) return;
  const int ntx = res_ntx(g, tx);
  const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
  const int t = threadIdx.x;
  const bool xtra = t >= tx * ty;
  if (xtra && !(bx == ntx - 1 && res_wide_last_x(g, tx))) return;
  const int x = bx * tx + (xtra ? tx : t % tx);
  const int y = by * ty + (xtra ? t - tx * ty : t / tx);
  if (x >= g.nn[0] || y >= g.nn[1]) return;
  const int i = ctrl->i_local;
  float* gi = (float*)Gown[i % 4];
  const float a0 = ctrl->alpha_f[0], a1 = ctrl->alpha_f[1], a2 = ctrl->alpha_f[2], a3 = ctrl->alpha_f[3];
  const float b0 = a0, b1 = a0 + a1, b2 = a0 + a1 + a2;
  const float* p0 = (const float*)P[(i - 3) % 4];
  const float* p1 = (const float*)P[(i - 2) % 4];
  const float* p2 = (const float*)P[(i - 1) % 4];
  const float* p3 = (const float*)P[i % 4];
  const float* r0 = (const float*)R[(i - 3) % 4];
  const float* r1 = (const float*)R[(i - 2) % 4];
  const float* r2 = (const float*)R[(i - 1) % 4];
  const float* g0 = (const float*)Gr[(i - 3) % 4];
  const float* g1 = (const float*)Gr[(i - 2) % 4];
  const float* g2 = (const float*)Gr[(i - 1) % 4];
  const int z0 = max(zr.x - 1, 0), z1 = min(zr.y + 1, g.nn[2] - 1);
  const long long plane = (long long)g.nn[0] * g.nn[1];
  for (int z = z0; z <= z1; ++z)
    for (int c = 0; c < 3; ++c) {
      const long long e = c * g.nnodes + plane * z + (long long)g.nn[0] * y + x;
      gi[e] = acv_combine(p0[e], p1[e], p2[e], p3[e], r0[e], r1[e], r2[e], g0[e], g1[e], g2[e], a0, a1, a2, a3, b0,
                          b1, b2);
    }
}

template <typename T>
int launch_acv_green_input(const GridDev& g, void* const* pring, void** gring, void* const* gown, void* const* rring,
                           const Ctrl* ctrl, int alias, const int2* tile_z, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  if constexpr (sizeof(T) == 4) {
    k_acv_green_input_v4<<<acv_blocks(g), SB, 0, s>>>(total, pring, gring, gown, rring, ctrl, alias);
    if (alias) {
      const int tx = residual_f32_tile(0), ty = residual_f32_tile(1);
      const int ntiles = res_ntx(g, tx) * ((g.nn[1] + ty - 1) / ty);
      k_acv_green_fix<<<ntiles, tx * ty + ty, 0, s>>>(g, pring, gring, gown, rring, ctrl, tile_z, tx, ty);
    }
  } else {
    k_acv_green_input<T><<<acv_blocks(g), SB, 0, s>>>(total, pring, gring, rring, ctrl);
  }
  return (int)cudaGetLastError();
}

// accelerate: x_i <- sum_m alpha_m (S_{j_m} + R_{j_m}), j_m = i-4+m.  ACV_P: the Green input
// becomes p + (x^ - x_i) (increment form); ACV_U: u~ is replaced and S_i = u~ stored.
template <typename T>
__global__ void k_acv_accel(long long total, int acv_on, void* const* S, void* const* R, T* gbuf,
                            double* u64, const Ctrl* ctrl) {
  if (ctrl->done) return;
  const int i = ctrl->i_local;
  const bool acc = ctrl->accel != 0;
  if (acv_on == 1 && !acc) return;
  const T *s0 = nullptr, *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;
  const T *r0 = nullptr, *r1 = nullptr, *r2 = nullptr, *r3 = nullptr;
  double al[4] = {0, 0, 0, 0};
  if (acc) {
    s0 = (const T*)S[(i - 4) % 5]; r0 = (const T*)R[(i - 4) % 4];
    s1 = (const T*)S[(i - 3) % 5]; r1 = (const T*)R[(i - 3) % 4];
    s2 = (const T*)S[(i - 2) % 5]; r2 = (const T*)R[(i - 2) % 4];
    s3 = (const T*)S[(i - 1) % 5]; r3 = (const T*)R[(i - 1) % 4];
    for (int m = 0; m < 4; ++m) al[m] = ctrl->alpha[m];
  }
  T* si = (T*)S[i % 5];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    if (acv_on == 1) {
      double xh = al[0] * ((double)s0[e] + (double)r0[e]) + al[1] * ((double)s1[e] + (double)r1[e]) +
                  al[2] * ((double)s2[e] + (double)r2[e]) + al[3] * ((double)s3[e] + (double)r3[e]);
      T xo = si[e];
      T xn = (T)xh;
      gbuf[e] = (T)((double)gbuf[e] + ((double)xn - (double)xo));
      si[e] = xn;
    } else {
      if (acc) {
        double v = al[0] * ((double)s0[e] + (double)r0[e]) + al[1] * ((double)s1[e] + (double)r1[e]) +
                   al[2] * ((double)s2[e] + (double)r2[e]) + al[3] * ((double)s3[e] + (double)r3[e]);
        u64[e] = v;
      }
      si[e] = (T)u64[e];
    }
  }
}

template <typename T>
int launch_acv_accel(const GridDev& g, int acv_on, void* const* Sring, void* const* Rring, T* gbuf,
                     double* u64, const Ctrl* ctrl, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  k_acv_accel<T><<<acv_blocks(g), SB, 0, s>>>(total, acv_on, Sring, Rring, gbuf, u64, ctrl);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ control
// Deterministic reduction of partial sums: fixed strided order + fixed tree.
// NV consecutive entries (off .. off + NV - 1) of n strided partial-sum records reduced in one
// pass: per thread in index order, then the warp shuffle tree, then warp totals in warp
// order -- the same order as NV separate reduce_fixed calls, with one barrier round.
// Results in out[0..NV-1] (shared memory, valid in every thread after the call).
template <int NV>
__device__ __forceinline__ void reduce_many(const double* v, int n, int stride, int off, double* out,
                                            double (*sh)[SB / 32]) {
  double acc[NV];
  #pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    #pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += v[(long long)k * stride + off + q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  #pragma unroll
  for (int q = 0; q < NV; ++q) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
  }
  __syncthreads();
  if (lane == 0)
    #pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][w] = acc[q];
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[threadIdx.x][k];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ double reduce_fixed(const double* v, int n, int stride, int off, double* sh) {
  double t = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) t += v[(long long)k * stride + off];
  double s = block_sum(t, sh);
  return s;
}

// Residual norms (Eq. 5), history and exit decision of one iteration (thread 0).
__device__ void ctrl_residual_core(Ctrl* c, double s2, double p2, double q2, double c2, double ng, double nr,
                                   double mm, double h, long long nnodes, long long nvox, double* hist) {
  double pt = p2 + q2 + c2;
  c->p2 = pt;
  c->s2 = s2;
  double pn = sqrt(pt / (double)nnodes), sn = sqrt(s2 / (double)nvox);
  double r = (sn == 0.0) ? (pn == 0.0 ? 0.0 : INFINITY) : h * pn / sn;
  c->r = r;
  if (c->iter == 0) {
    c->r0 = r;
    c->pn0 = pn;
  }
  if (c->hist_len < HIST) hist[c->hist_len++] = r;
  c->pslot = c->i_local % 4;
  c->n_vgap = (int)ng;
  c->n_vreact = (int)nr;
  c->n_mismatch = (int)mm;
  c->update = 0;
  c->changed = 0;
  const bool sets_empty = (c->n_vgap == 0 && c->n_vreact == 0);
  if (c->no_stop) return;
  if (r < c->tol && (!c->contact_on || sets_empty)) { c->done = 1; return; }
  if (c->iter >= c->max_iter) { c->done = 2; return; }
  // Divergence.  Eq. 5 scales ||p|| by ||sigma||, and an unstable mode grows both, so r
  // alone stays O(1) while the iterate blows up; the RMS of p is watched as well.
  if (!isfinite(r) || (c->r0 > 0.0 && r > 1e6 * c->r0) || (c->pn0 > 0.0 && pn > 1e6 * c->pn0)) {
    c->done = 3;
    return;
  }
  if (c->contact_on) {
    if (c->prev_valid && c->n_mismatch == 0 && r < c->update_tol) c->update = 1;
    c->prev_valid = 1;
  }
}

__global__ void k_ctrl_residual(Ctrl* c, const double* rp, int nres, const double* pp, int nproj,
                                const double* cp, int ncont, double h, long long nnodes, long long nvox) {
  __shared__ double sh[SB / 32];
  if (c->done) return;
  double s2 = reduce_fixed(rp, nres, RES_STRIDE, 0, sh);
  double p2 = reduce_fixed(rp, nres, RES_STRIDE, 1, sh);
  double q2 = (nproj > 0) ? reduce_fixed(pp, nproj, PROJ_STRIDE, 0, sh) : 0.0;
  double c2 = 0.0, ng = 0.0, nr = 0.0, mm = 0.0;
  if (ncont > 0) {
    c2 = reduce_fixed(cp, ncont, CONT_STRIDE, 0, sh);
    ng = reduce_fixed(cp, ncont, CONT_STRIDE, 1, sh);
    nr = reduce_fixed(cp, ncont, CONT_STRIDE, 2, sh);
    mm = reduce_fixed(cp, ncont, CONT_STRIDE, 3, sh);
  }
  if (threadIdx.x != 0) return;
  ctrl_residual_core(c, s2, p2, q2, c2, ng, nr, mm, h, nnodes, nvox, c->hist);
}

__global__ void k_ctrl_contact(Ctrl* c) {
  if (c->done) return;
  if (c->changed > 0) {
    c->i_local = 0;
    c->n_updates += 1;
  }
}

int launch_ctrl_contact(Ctrl* c, cudaStream_t s) {
  k_ctrl_contact<<<1, 1, 0, s>>>(c);
  return (int)cudaGetLastError();
}

// Gram update of slot (i-1) % 4 and, every acv_mod iterations after the first four, the
// constrained least squares for alpha (thread 0).
__device__ __forceinline__ void ctrl_acv_core(Ctrl* c, const double* d) {
  const int i = c->i_local;
  c->accel = 0;
  if (i > 0) {
    int s = (i - 1) % 4;
    for (int k = 0; k < 4; ++k) { c->gram[s][k] = d[k]; c->gram[k][s] = d[k]; }
  }
  if (i >= 4 && (i % c->acv_mod) == 0) {
    double A[4][4], b[4] = {1, 1, 1, 1};
    double scale = 0.0;
    for (int r = 0; r < 4; ++r) {
      for (int q = 0; q < 4; ++q) A[r][q] = c->gram[r][q];
      scale = fmax(scale, fabs(A[r][r]));
    }
    bool ok = scale > 0.0;
    for (int col = 0; col < 4 && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < 4; ++r)
        if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      if (fabs(A[piv][col]) <= c->acv_pivot * scale) { ok = false; break; }
      if (piv != col) {
        for (int q = 0; q < 4; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        double t = b[col]; b[col] = b[piv]; b[piv] = t;
      }
      for (int r = col + 1; r < 4; ++r) {
        double m = A[r][col] / A[col][col];
        for (int q = col; q < 4; ++q) A[r][q] -= m * A[col][q];
        b[r] -= m * b[col];
      }
    }
    if (ok) {
      double y[4];
      for (int r = 3; r >= 0; --r) {
        double t = b[r];
        for (int q = r + 1; q < 4; ++q) t -= A[r][q] * y[q];
        y[r] = t / A[r][r];
      }
      double sy = y[0] + y[1] + y[2] + y[3];
      if (sy != 0.0 && isfinite(sy)) {
        for (int m = 0; m < 4; ++m) {
          c->alpha[m] = y[(i - 4 + m) % 4] / sy;
          c->alpha_f[m] = (float)c->alpha[m];
        }
        c->accel = 1;
        c->n_accel += 1;
      }
    }
  }
}

__global__ void k_ctrl_acv(Ctrl* c, const double* partials, int nblk) {
  __shared__ double sh[SB / 32];
  if (c->done) return;
  __shared__ double d[4];   // Gram row, written and read by thread 0
  const int i = c->i_local;
  #pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double t = (i > 0) ? reduce_fixed(partials, nblk, 4, k, sh) : 0.0;
    if (threadIdx.x == 0) d[k] = t;
  }
  if (threadIdx.x != 0) return;
  ctrl_acv_core(c, d);
}

__global__ void k_ctrl_acv_fused(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, const double* cp,
                                 int ncont) {
  __shared__ double sh[SB / 32];
  if (c->done) return;
  __shared__ double d[4];   // Gram row, written and read by thread 0
  const int i = c->i_local;
  #pragma unroll
  for (int k = 0; k < 4; ++k) {
    double t = 0.0;
    if (i > 0) {
      t = reduce_fixed(rp, nres, RES_STRIDE, 2 + k, sh);
      if (nproj > 0) t += reduce_fixed(pp, nproj, PROJ_STRIDE, 1 + k, sh);
      if (ncont > 0) t += reduce_fixed(cp, ncont, CONT_STRIDE, 4 + k, sh);
    }
    if (threadIdx.x == 0) d[k] = t;
  }
  if (threadIdx.x != 0) return;
  ctrl_acv_core(c, d);
}

// k_ctrl_residual followed by k_ctrl_acv_fused in one launch (iterations without contact,
// where nothing runs between the two); both reductions in one pass each.  The control
// state except the residual history is staged in shared memory by one parallel copy, so
// that thread 0's sequential logic (the Eq. 5 test, the Gram update, the 4 x 4 solve) does
// not wait on a global-memory round trip per field; it is written back the same way.
constexpr int CTRL_HEAD_WORDS = (int)(offsetof(Ctrl, hist) / sizeof(double));
static_assert(offsetof(Ctrl, hist) % sizeof(double) == 0, "Ctrl head must be a whole number of doubles");

__global__ void k_ctrl_residual_acv(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, double h,
                                    long long nnodes, long long nvox) {
  __shared__ double sh[RES_STRIDE][SB / 32];
  __shared__ double rs[RES_STRIDE], ps[PROJ_STRIDE];
  __shared__ double d[4];   // Gram row (thread 0)
  __shared__ int sdone;
  __shared__ double head[CTRL_HEAD_WORDS];
  for (int q = threadIdx.x; q < CTRL_HEAD_WORDS; q += blockDim.x) head[q] = ((const double*)c)[q];
  __syncthreads();
  Ctrl* sc = (Ctrl*)head;   // only members before the history are touched through sc
  if (sc->done) return;
  reduce_many<RES_STRIDE>(rp, nres, RES_STRIDE, 0, rs, sh);   // [s2, p2, Gram 0..3]
  if (nproj > 0) {
    reduce_many<PROJ_STRIDE>(pp, nproj, PROJ_STRIDE, 0, ps, sh);   // [p2, Gram 0..3]
  } else if (threadIdx.x < PROJ_STRIDE) {
    ps[threadIdx.x] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl_residual_core(sc, rs[0], rs[1], ps[0], 0.0, 0.0, 0.0, 0.0, h, nnodes, nvox, c->hist);
    sdone = sc->done;
    if (!sdone) {
      const bool row = sc->i_local > 0;
      for (int k = 0; k < 4; ++k) d[k] = row ? rs[2 + k] + ps[1 + k] : 0.0;
      ctrl_acv_core(sc, d);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < CTRL_HEAD_WORDS; q += blockDim.x) ((double*)c)[q] = head[q];
}

int launch_ctrl_residual_acv(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, double h,
                             long long nnodes, long long nvox, cudaStream_t s) {
  k_ctrl_residual_acv<<<1, SB, 0, s>>>(c, rp, nres, pp, nproj, h, nnodes, nvox);
  return (int)cudaGetLastError();
}

int launch_ctrl_acv_fused(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, const double* cp,
                          int ncont, cudaStream_t s) {
  k_ctrl_acv_fused<<<1, SB, 0, s>>>(c, rp, nres, pp, nproj, cp, ncont);
  return (int)cudaGetLastError();
}

int launch_ctrl_acv(Ctrl* c, const double* partials, int nblk, cudaStream_t s) {
  k_ctrl_acv<<<1, SB, 0, s>>>(c, partials, nblk);
  return (int)cudaGetLastError();
}

__global__ void k_ctrl_end(Ctrl* c) {
  if (c->done) return;
  c->iter += 1;
  c->i_local += 1;
}

int launch_ctrl_end(Ctrl* c, cudaStream_t s) {
  k_ctrl_end<<<1, 1, 0, s>>>(c);
  return (int)cudaGetLastError();
}

// residual control: partial regions of the residual (2 per block), row projection (1 per
// block) and contact (4 per block) kernels
int launch_ctrl_residual(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, const double* cp,
                          int ncont, double h, long long nnodes, long long nvox, cudaStream_t s) {
  k_ctrl_residual<<<1, SB, 0, s>>>(c, rp, nres, pp, nproj, cp, ncont, h, nnodes, nvox);
  return (int)cudaGetLastError();
}

template int launch_proj_P_rows<double>(const GridDev&, const RowsDev&, double*, void* const*, void* const*, int, int, double*, const Ctrl*, cudaStream_t, double*);
template int launch_proj_P_rows<float>(const GridDev&, const RowsDev&, float*, void* const*, void* const*, int, int, double*, const Ctrl*, cudaStream_t, float*);
template int launch_proj_U_rows<double>(const GridDev&, const RowsDev&, double*, float*, float*, double*, const Ctrl*, cudaStream_t);
template int launch_proj_U_rows<float>(const GridDev&, const RowsDev&, double*, float*, float*, float*, const Ctrl*, cudaStream_t);
template int launch_proj_U_rows_end<double>(const GridDev&, const RowsDev&, double*, float*, float*, double*, Ctrl*, cudaStream_t);
template int launch_proj_U_rows_end<float>(const GridDev&, const RowsDev&, double*, float*, float*, float*, Ctrl*, cudaStream_t);
template int launch_contact_eval<double>(const ContactArgs&, double*, void* const*, void* const*, int, int, cudaStream_t);
template int launch_contact_eval<float>(const ContactArgs&, float*, void* const*, void* const*, int, int, cudaStream_t);
template int launch_contact_proj_U<double>(const ContactArgs&, double*, float*, float*, double*, cudaStream_t);
template int launch_contact_proj_U<float>(const ContactArgs&, double*, float*, float*, float*, cudaStream_t);
template int launch_acv_gram<double>(const GridDev&, void* const*, double*, const Ctrl*, cudaStream_t);
template int launch_acv_gram<float>(const GridDev&, void* const*, double*, const Ctrl*, cudaStream_t);
template int launch_acv_green_input<double>(const GridDev&, void* const*, void**, void* const*, void* const*, const Ctrl*,
                                            int, const int2*, cudaStream_t);
template int launch_acv_green_input<float>(const GridDev&, void* const*, void**, void* const*, void* const*, const Ctrl*,
                                           int, const int2*, cudaStream_t);
template int launch_acv_store<double>(const GridDev&, int, void* const*, void* const*, const double*, double*, const Ctrl*, cudaStream_t);
template int launch_acv_store<float>(const GridDev&, int, void* const*, void* const*, const double*, double*, const Ctrl*, cudaStream_t);
template int launch_acv_accel<double>(const GridDev&, int, void* const*, void* const*, double*, double*, const Ctrl*, cudaStream_t);
template int launch_acv_accel<float>(const GridDev&, int, void* const*, void* const*, float*, double*, const Ctrl*, cudaStream_t);

__global__ void k_batch_done(Ctrl* const* ctrls, int n, int* done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) done[i] = ctrls[i]->done;
}

// Condition of the device-side solve loop (a conditional WHILE node of the solve's CUDA
// graph around `iters` captured iterations): run another round while any of the grids
// (ctrls[0..n), or the single control block `one`) is still iterating and fewer than
// rounds[1] rounds have run (rounds[0] counts them; the cap only guards the loop, each grid
// stops at its max_iter).  max_rounds > 0 overrides rounds[1].
__global__ void k_loop_continue(Ctrl* const* ctrls, const Ctrl* one, int n, cudaGraphConditionalHandle h,
                                int* rounds, int max_rounds) {
  __shared__ int running;
  if (threadIdx.x == 0) running = one ? !one->done : 0;
  __syncthreads();
  if (!one)
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (!ctrls[i]->done) atomicOr(&running, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int r = rounds[0] + 1;
    rounds[0] = r;
    const int cap = max_rounds > 0 ? max_rounds : rounds[1];
    cudaGraphSetConditional(h, (running && r < cap) ? 1u : 0u);
  }
}

int launch_loop_continue(Ctrl* const* ctrls, const Ctrl* one, int n, cudaGraphConditionalHandle h, int* rounds,
                         int max_rounds, cudaStream_t s) {
  k_loop_continue<<<1, 256, 0, s>>>(ctrls, one, n, h, rounds, max_rounds);
  return (int)cudaGetLastError();
}

int launch_batch_done(Ctrl* const* ctrls, int n, int* done, cudaStream_t s) {
  if (n <= 0) return 0;
  k_batch_done<<<(n + 255) / 256, 256, 0, s>>>(ctrls, n, done);
  return (int)cudaGetLastError();
}

}  // namespace dtt

// Per-axis discrete trigonometric transforms, the Green multiply and the increment update
// (Algorithm 1: DT(p) -> p^, u^ = G_D(p^), iDT(u^) -> u~).
//
// Transform choice per component and axis (Section 3.2.2, Tables 2-3): SS -> DCT1 on
// nodes [0:n], SA -> DCT3 on [0:n-1], AA -> DST1 on [1:n-1], AS -> DST3 on [1:n], wave
// numbers q_k = pi k/n (DCT1, DST1) or pi(2k+1)/(2n) (DCT3, DST3).  A periodic axis uses
// the discrete Hartley transform (cas = cos + sin, q_k = 2 pi k/n): the Green symbol is
// even in each q, so the real Hartley basis diagonalises the operator exactly as the
// complex DFT does, and every spectrum stays real.
//
// Each axis pass is a batched dense contraction out = M * in along that axis, M being the
// (nn x nn) transform matrix of the component (zero rows/columns outside the selection),
// tiled through shared memory: for the y and z axes the contiguous x index is the GEMM's
// N dimension (coalesced); for the x axis the pencil index is M and the matrix is applied
// from the right.  The Green multiply divides each spectral value by
//     a_c(q) = lambda0 S_c(q) + 2 mu0 (S_x + S_y + S_z)
// (TETRA2: S_j = (1 + c_k c_l - c_j c_k - c_j c_l)/h^2; HEX1: S_j = (1-c_j)(1+c_k)(1+c_l)/(2h^2),
// c_j = cos q_j; evaluated through sin^2(q_j/2) and cos^2(q_j/2)), zeroing null modes
// (a_c <= threshold).
#include <algorithm>

#include "dtt_internal.cuh"

namespace dtt {

constexpr int GBM = 64, GBN = 64, GBK = 16;

// out[o][m][n] = sum_k A[m][k] * in[o][k][n];  A: len x len, in/out slabs len x inner.
template <typename T>
__global__ void __launch_bounds__(256)
k_axis_left(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ A0m,
            const T* __restrict__ A1m, const T* __restrict__ A2m, int len, int inner, int outer,
            long long NN, int comp0, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  __shared__ T As[GBK][GBM + 1];
  __shared__ T Bs[GBK][GBN];
  const int comp = comp0 + blockIdx.z / outer;
  const int o = blockIdx.z % outer;
  const T* A = comp == 0 ? A0m : (comp == 1 ? A1m : A2m);
  const T* B = in + (long long)comp * NN + (long long)o * len * inner;
  T* C = out + (long long)comp * NN + (long long)o * len * inner;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
  #pragma unroll
  for (int i = 0; i < 4; ++i)
    #pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int k0 = 0; k0 < len; k0 += GBK) {
    for (int q = threadIdx.x; q < GBM * GBK; q += 256) {
      int mm = q / GBK, kk = q % GBK;
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < len && gk < len) ? A[(long long)gm * len + gk] : (T)0;
    }
    for (int q = threadIdx.x; q < GBK * GBN; q += 256) {
      int kk = q / GBN, nn = q % GBN;
      int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < len && gn < inner) ? B[(long long)gk * inner + gn] : (T)0;
    }
    __syncthreads();
    #pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      T a[4], b[4];
      #pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
      #pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
      #pragma unroll
      for (int i = 0; i < 4; ++i)
        #pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  #pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= len) continue;
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn < inner) C[(long long)gm * inner + gn] = acc[i][j];
    }
  }
}

// out[r][n] = sum_k in[r][k] * A[n][k];  rows r = pencils along x (len contiguous).
template <typename T>
__global__ void __launch_bounds__(256)
k_axis_right(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ A0m,
             const T* __restrict__ A1m, const T* __restrict__ A2m, int len, int rows, long long NN,
             int comp0, const Ctrl* ctrl, void* const* in_ring) {
  if (ctrl && ctrl->done) return;
  if (in_ring) in = (const T*)in_ring[ctrl->i_local % 4];
  __shared__ T As[GBK][GBM + 1];   // pencil rows (k, r)
  __shared__ T Bs[GBK][GBN + 1];   // matrix (k, n)
  const int comp = comp0 + blockIdx.z;
  const T* A = comp == 0 ? A0m : (comp == 1 ? A1m : A2m);
  const T* X = in + (long long)comp * NN;
  T* C = out + (long long)comp * NN;
  const int r0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
  #pragma unroll
  for (int i = 0; i < 4; ++i)
    #pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int k0 = 0; k0 < len; k0 += GBK) {
    for (int q = threadIdx.x; q < GBM * GBK; q += 256) {
      int rr = q / GBK, kk = q % GBK;
      int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < rows && gk < len) ? X[(long long)gr * len + gk] : (T)0;
    }
    for (int q = threadIdx.x; q < GBN * GBK; q += 256) {
      int nn = q / GBK, kk = q % GBK;
      int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < len && gk < len) ? A[(long long)gn * len + gk] : (T)0;
    }
    __syncthreads();
    #pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      T a[4], b[4];
      #pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
      #pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
      #pragma unroll
      for (int i = 0; i < 4; ++i)
        #pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  #pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gr = r0 + ty + 16 * i;
    if (gr >= rows) continue;
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn < len) C[(long long)gr * len + gn] = acc[i][j];
    }
  }
}

static FftParams fft_params(const GridDev& g, const TransformTables& tt, int axis, int inverse, int ncomp_first) {
  const FftAxisInfo& fa = tt.fft[axis];
  FftParams p{};
  p.axis = axis;
  p.n = g.nvox[axis];
  p.nn = g.nn[axis];
  p.L = fa.L;
  p.nst = fa.nst;
  for (int q = 0; q < 12; ++q) p.radix[q] = fa.radix[q];
  p.tw = fa.tw;
  p.ph = fa.ph;
  for (int c = 0; c < 3; ++c) p.type[c] = tt.types[c][axis];
  p.inverse = inverse;
  p.comp0 = ncomp_first;
  p.nnx = g.nn[0];
  p.nny = g.nn[1];
  p.NN = g.nnodes;
  p.npencil = g.nnodes / g.nn[axis];
  p.scale = 1.0;
  if (inverse) p.scale = g.periodic[axis] ? 1.0 / g.nvox[axis] : 2.0 / g.nvox[axis];
  p.fscale = (float)p.scale;
  p.generic = g.fft_generic;
  p.inv_n = 1.0 / g.nvox[axis];
  p.finv_n = (float)p.inv_n;
  return p;
}

template <typename T>
int launch_z_green(const GridDev& g, const T* in, T* out, const TransformTables& tt, int ncomp_first, int ncomp,
                   const Ctrl* ctrl, cudaStream_t s) {
  if (!tt.fft[2].use && !(sizeof(T) == 4 && tt.tz_use)) return (int)cudaErrorInvalidValue;
  FftParams p = fft_params(g, tt, 2, 0, ncomp_first);
  GreenTables gt;
  for (int c = 0; c < 3; ++c) {
    for (int d = 0; d < 3; ++d) {
      gt.s[c][d] = tt.sin2q[c][d];
      gt.cp[c][d] = tt.cos2q[c][d];
      gt.sf[c][d] = tt.sin2q_f[c][d];
      gt.cpf[c][d] = tt.cos2q_f[c][d];
    }
    gt.null_thr[c] = tt.null_thr[c];
    gt.null_thr_f[c] = (float)tt.null_thr[c];
  }
  if constexpr (sizeof(T) == 4) {
    if (tt.tz_use) {
      TzParams tp{};
      for (int c = 0; c < 3; ++c) tp.c[c] = tt.tz[c];
      tp.comp0 = ncomp_first;
      tp.nnx = g.nn[0];
      tp.nnz = g.nn[2];
      tp.NN = g.nnodes;
      tp.stride = (long long)g.nn[0] * g.nn[1];
      tp.npencil = tp.stride;
      tp.err = tt.tz_err;
      return launch_tz_green((const float*)in, (float*)out, tp, gt, tt.lam0, tt.mu0, g.scheme, g.h, ncomp, ctrl, s);
    }
  }
  return launch_fft_z_green<T>(in, out, p, gt, tt.lam0, tt.mu0, g.scheme, g.h, ncomp, ctrl, s);
}

template <typename T>
int launch_transform_axis(const GridDev& g, const T* in, T* out, const TransformTables& tt,
                          int axis, int inverse, int ncomp_first, int ncomp, const Ctrl* ctrl,
                          cudaStream_t s, void* const* in_ring, const IncrTarget* incr) {
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];
  if (tt.fft[axis].use) {
    FftParams p = fft_params(g, tt, axis, inverse, ncomp_first);
    if (incr) {
      if (axis != 0 || !inverse) return (int)cudaErrorInvalidValue;
      p.incr = 1;
      p.u64 = incr->u64;
      p.uhi = incr->uhi;
      p.ulo = incr->ulo;
      p.step = incr->step;
    }
    return launch_fft_axis<T>(in, out, p, ncomp, ctrl, in_ring, s);
  }
  if (incr) return (int)cudaErrorInvalidValue;
  {
    FftParams p;
    (void)p;
  }
  const T* M[3];
  for (int c = 0; c < 3; ++c)
    M[c] = (const T*)(inverse ? tt.inv[c][axis] : tt.fwd[c][axis]);
  if (axis == 0) {
    int rows = nny * nnz;
    dim3 grd((nnx + GBN - 1) / GBN, (rows + GBM - 1) / GBM, ncomp);
    k_axis_right<T><<<grd, 256, 0, s>>>(in, out, M[0], M[1], M[2], nnx, rows, g.nnodes, ncomp_first, ctrl, in_ring);
  } else {
    if (in_ring) return (int)cudaErrorInvalidValue;   // ring input only on the first (x) pass
    int len = axis == 1 ? nny : nnz;
    int inner = axis == 1 ? nnx : nnx * nny;
    int outer = axis == 1 ? nnz : 1;
    dim3 grd((inner + GBN - 1) / GBN, (len + GBM - 1) / GBM, outer * ncomp);
    k_axis_left<T><<<grd, 256, 0, s>>>(in, out, M[0], M[1], M[2], len, inner, outer, g.nnodes, ncomp_first, ctrl);
  }
  return (int)cudaGetLastError();
}

// s_j = sin^2(q_j/2) and c'_j = cos^2(q_j/2) (tables exact in double) keep the symbol
// accurate both near q = 0 and near the checkerboard q = (pi,pi,pi), where the plain
// cosine form cancels:  TETRA2  S_x / 4 = s_x c'_y + s_z (s_y - s_x),  s_y - s_x = c'_x - c'_y;
//                       HEX1    S_x / 4 = s_x c'_y c'_z.
template <typename T>
__device__ __forceinline__ T tetra_S(T sa, T cb, T sb, T cA, T sc) {
  // S_a / 4 = s_a c'_b + s_c (s_b - s_a), difference taken in the accurate variables
  const T d = (sa + sb < (T)1) ? (sb - sa) : (cA - cb);
  return sa * cb + sc * d;
}

template <typename T>
__global__ void k_green(const GridDev g, T* __restrict__ spec, GreenTables gt, double lam0, double mu0,
                        const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  // grid: x = x-index blocks, y = y index, z = component * nn_z + z index
  const int c = blockIdx.z / g.nn[2];
  const int k = blockIdx.z - c * g.nn[2];
  const int j = blockIdx.y;
  const T ih2 = (T)(4.0 / (g.h * g.h));
  const T sy = gt_s<T>(gt, c, 1, j), sz = gt_s<T>(gt, c, 2, k);
  const T cy = gt_c<T>(gt, c, 1, j), cz = gt_c<T>(gt, c, 2, k);
  const T l0 = (T)lam0, m2 = (T)(2.0 * mu0), thr = sizeof(T) == 4 ? (T)gt.null_thr_f[c] : (T)gt.null_thr[c];
  T* row = spec + (long long)c * g.nnodes + ((long long)k * g.nn[1] + j) * g.nn[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nn[0]; i += gridDim.x * blockDim.x) {
    const T sx = gt_s<T>(gt, c, 0, i), cx = gt_c<T>(gt, c, 0, i);
    T Sx, Sy, Sz;
    if (g.scheme == SCHEME_TETRA2) {
      Sx = tetra_S<T>(sx, cy, sy, cx, sz);
      Sy = tetra_S<T>(sy, cz, sz, cy, sx);
      Sz = tetra_S<T>(sz, cx, sx, cz, sy);
    } else {
      Sx = sx * cy * cz;
      Sy = sy * cx * cz;
      Sz = sz * cx * cy;
    }
    const T Sc = c == 0 ? Sx : (c == 1 ? Sy : Sz);
    const T a = (l0 * Sc + m2 * (Sx + Sy + Sz)) * ih2;
    row[i] = (a <= thr) ? (T)0 : row[i] / a;
  }
}

template <typename T>
int launch_green_multiply(const GridDev& g, T* spec, const TransformTables& tt, int scheme,
                          const Ctrl* ctrl, cudaStream_t s) {
  (void)scheme;
  GreenTables gt;
  for (int c = 0; c < 3; ++c) {
    for (int d = 0; d < 3; ++d) {
      gt.s[c][d] = tt.sin2q[c][d];
      gt.cp[c][d] = tt.cos2q[c][d];
      gt.sf[c][d] = tt.sin2q_f[c][d];
      gt.cpf[c][d] = tt.cos2q_f[c][d];
    }
    gt.null_thr[c] = tt.null_thr[c];
    gt.null_thr_f[c] = (float)tt.null_thr[c];
  }
  dim3 grd((g.nn[0] + 127) / 128, g.nn[1], 3 * g.nn[2]);
  k_green<T><<<grd, 128, 0, s>>>(g, spec, gt, tt.lam0, tt.mu0, ctrl);
  return (int)cudaGetLastError();
}

// Green step of the isotropic reference medium R0 : grad u = lambda0 tr(grad u) 1 +
// mu0 (grad u + grad u^T) (Section 3.2.3; Eq. 4 for HEX1 in the periodic case).  With
// normal mixed conditions on the non-periodic axes, every component's DTT basis function
// of wave vector q is mapped by A0 onto the same q of every component along those axes.
// Along a periodic axis the basis is the Hartley cas(q x), and a first difference maps
// cas(q x) onto cas(-q x): the cross term of components c and d flips the wave numbers of
// the periodic axes among {c, d}.  Those flips compose, so u_x at position q, u_y at q
// flipped on the periodic axes of {x, y} and u_z at q flipped on those of {x, z} form a
// closed symmetric 3 x 3 system:
//     M_cc = (lambda0 + mu0) S_c + mu0 (S_x + S_y + S_z),
//     M_cd = sign_c sign_d tau_cd (lambda0 + mu0) T_cd        (c != d),
// with the scheme's S_j (as in k_green; even in every q, so the same at the three
// positions), the cross symbols
//     TETRA2: T_cd = sin q_c sin q_d / h^2,  HEX1: T_cd = sin q_c sin q_d cos^2(q_e / 2) / h^2
// (e the third axis; both from the schemes' gradients, and real because both stencils are
// centrosymmetric) taken at the x component's position q with signed sines on the
// periodic axes, sign_d = +1 when the normal component's transform along d is a sine
// transform and -1 otherwise (a periodic axis counts as -1), and tau_cd = -1 for the pairs
// (x, y), (x, z) when the x axis is periodic, +1 otherwise.  (Rule checked against the
// operator's spectral matrix, entry by entry, for every periodic pattern and both
// schemes.)  In the quarter units of the tables (4 / h^2 factored out):
// |sin q_c sin q_d| / 4 = sqrt(s_c c'_c s_d c'_d).  A component without a mode at its
// position, or whose diagonal vanishes (a null mode, where all its cross terms vanish too),
// keeps a zero coefficient; the rest is solved by LDL^T (symmetric positive definite).
// Each thread takes the triple of one x position; the flips are bijections, so every
// position of every component belongs to exactly one triple.
// The scalar constants come from the host (ih2 = 4 / h^2, ih2r = its inverse, lm = lambda0 +
// mu0, m0 = mu0, thr the null threshold): no per-thread FP64 arithmetic.
template <typename T>
__global__ void k_green_iso(const GridDev g, T* __restrict__ spec, IsoTables it, T ih2, T ih2r, T lm, T m0, T thr,
                            const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  const long long NN = g.nnodes;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < NN; n += (long long)gridDim.x * blockDim.x) {
    // position on the node grid; 32-bit division when the grid allows it (64-bit integer
    // division is a long software sequence)
    int i, j, k;
    if (NN <= 0x7fffffffLL) {
      const int n32 = (int)n, r = n32 / g.nn[0];
      i = n32 - r * g.nn[0];
      j = r % g.nn[1];
      k = r / g.nn[1];
    } else {
      const long long r = n / g.nn[0];
      i = (int)(n - r * g.nn[0]);
      j = (int)(r % g.nn[1]);
      k = (int)(r / g.nn[1]);
    }
    const int valid = it.valid[0][i] & it.valid[1][j] & it.valid[2][k];
    // positions of the triple: flips on the periodic axes of {x, y} (y) and {x, z} (z)
    const int fi = g.periodic[0] ? (i == 0 ? 0 : g.nn[0] - i) : i;
    const int fj = g.periodic[1] ? (j == 0 ? 0 : g.nn[1] - j) : j;
    const int fk = g.periodic[2] ? (k == 0 ? 0 : g.nn[2] - k) : k;
    const long long np[3] = {n, fi + (long long)g.nn[0] * (fj + (long long)g.nn[1] * k),
                             fi + (long long)g.nn[0] * (j + (long long)g.nn[1] * fk)};
    // sign of sin q at the x position: + on a non-periodic axis (q in [0, pi]); on a
    // periodic axis + for 0 < p < n/2, - for p > n/2 (0 where sin q = 0)
    const int pidx[3] = {i, j, k};
    T ssg[3];
    #pragma unroll
    for (int d = 0; d < 3; ++d) ssg[d] = (g.periodic[d] && 2 * pidx[d] > g.nn[d]) ? (T)-1 : (T)1;
    T sv[3], cv[3];
    const int pos[3] = {i, j, k};
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (sizeof(T) == 4) { sv[d] = it.sf[d][pos[d]]; cv[d] = it.cf[d][pos[d]]; }
      else { sv[d] = (T)it.s[d][pos[d]]; cv[d] = (T)it.c[d][pos[d]]; }
    }
    T S[3];
    if (g.scheme == SCHEME_TETRA2) {
      S[0] = tetra_S<T>(sv[0], cv[1], sv[1], cv[0], sv[2]);
      S[1] = tetra_S<T>(sv[1], cv[2], sv[2], cv[1], sv[0]);
      S[2] = tetra_S<T>(sv[2], cv[0], sv[0], cv[2], sv[1]);
    } else {
      S[0] = sv[0] * cv[1] * cv[2];
      S[1] = sv[1] * cv[0] * cv[2];
      S[2] = sv[2] * cv[0] * cv[1];
    }
    T rt[3];   // sqrt(s c'): sin q / 2
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
      if constexpr (sizeof(T) == 4) rt[d] = sqrtf(sv[d] * cv[d]);
      else rt[d] = sqrt(sv[d] * cv[d]);
    }
    const T Ssum = S[0] + S[1] + S[2];
    T M[3][3], b[3];
    bool on[3];
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
      M[c][c] = lm * S[c] + m0 * Ssum;
      on[c] = ((valid >> c) & 1) && M[c][c] * ih2 > thr;
      b[c] = on[c] ? spec[(long long)c * NN + np[c]] : (T)0;
    }
    #pragma unroll
    for (int c = 0; c < 3; ++c)
      #pragma unroll
      for (int d = c + 1; d < 3; ++d) {
        const int e = 3 - c - d;
        T t = (rt[c] * ssg[c]) * (rt[d] * ssg[d]);
        if (g.scheme != SCHEME_TETRA2) t *= cv[e];
        const int tau = (g.periodic[0] && c == 0) ? -1 : 1;   // pairs (x, y), (x, z) when x is periodic
        t *= (T)(it.sign[c] * it.sign[d] * tau) * lm;
        if (!on[c] || !on[d]) t = (T)0;
        M[c][d] = t;
        M[d][c] = t;
      }
    #pragma unroll
    for (int c = 0; c < 3; ++c)
      if (!on[c]) M[c][c] = (T)1;
    // LDL^T of the symmetric positive definite M, then the two triangular solves
    const T r0 = (T)1 / M[0][0];
    const T L10 = M[1][0] * r0, L20 = M[2][0] * r0;
    const T D1 = M[1][1] - L10 * M[1][0];
    const T r1 = (T)1 / D1;
    const T L21 = (M[2][1] - L20 * M[1][0]) * r1;
    const T D2 = M[2][2] - L20 * M[2][0] - L21 * L21 * D1;
    const T r2 = (T)1 / D2;
    const T y0 = b[0], y1 = b[1] - L10 * y0, y2 = b[2] - L20 * y0 - L21 * y1;
    const T x2 = y2 * r2;
    const T x1 = y1 * r1 - L21 * x2;
    const T x0 = y0 * r0 - L10 * x1 - L20 * x2;
    const T x[3] = {x0, x1, x2};
    #pragma unroll
    for (int c = 0; c < 3; ++c) spec[(long long)c * NN + np[c]] = on[c] ? x[c] * ih2r : (T)0;
  }
}

template <typename T>
int launch_green_iso(const GridDev& g, T* spec, const TransformTables& tt, const Ctrl* ctrl, cudaStream_t s) {
  const long long nb = std::min<long long>((g.nnodes + 255) / 256, 148LL * 16);
  const double h2 = g.h * g.h;
  k_green_iso<T><<<(int)nb, 256, 0, s>>>(g, spec, tt.iso, (T)(4.0 / h2), (T)(h2 / 4.0), (T)(tt.lam0 + tt.mu0),
                                         (T)tt.mu0, (T)tt.iso.null_thr, ctrl);
  return (int)cudaGetLastError();
}

template int launch_green_iso<double>(const GridDev&, double*, const TransformTables&, const Ctrl*, cudaStream_t);
template int launch_green_iso<float>(const GridDev&, float*, const TransformTables&, const Ctrl*, cudaStream_t);

// u~ <- u~ + delta (Green step in increment form: G(p~) = u~ + G(p~ - A0 u~)).
template <typename T>
__global__ void k_add_increment(long long total, const T* __restrict__ delta, double* __restrict__ u64,
                                float* __restrict__ uhi, float* __restrict__ ulo, T* __restrict__ step,
                                const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    if (step) step[e] = delta[e];
    if constexpr (sizeof(T) == 8) {
      u64[e] += (double)delta[e];
    } else {
      float h = uhi[e], l = ulo[e];
      ff_add(h, l, (float)delta[e]);
      uhi[e] = h;
      ulo[e] = l;
    }
  }
}

template <typename T>
int launch_add_increment(const GridDev& g, const T* delta, double* u64, float* uhi, float* ulo,
                         T* step_out, const Ctrl* ctrl, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
  k_add_increment<T><<<blocks, 256, 0, s>>>(total, delta, u64, uhi, ulo, step_out, ctrl);
  return (int)cudaGetLastError();
}

template int launch_transform_axis<double>(const GridDev&, const double*, double*, const TransformTables&, int, int, int, int, const Ctrl*, cudaStream_t, void* const*, const IncrTarget*);
template int launch_transform_axis<float>(const GridDev&, const float*, float*, const TransformTables&, int, int, int, int, const Ctrl*, cudaStream_t, void* const*, const IncrTarget*);
template int launch_z_green<double>(const GridDev&, const double*, double*, const TransformTables&, int, int, const Ctrl*, cudaStream_t);
template int launch_z_green<float>(const GridDev&, const float*, float*, const TransformTables&, int, int, const Ctrl*, cudaStream_t);
template int launch_green_multiply<double>(const GridDev&, double*, const TransformTables&, int, const Ctrl*, cudaStream_t);
template int launch_green_multiply<float>(const GridDev&, float*, const TransformTables&, int, const Ctrl*, cudaStream_t);
template int launch_add_increment<double>(const GridDev&, const double*, double*, float*, float*, double*, const Ctrl*, cudaStream_t);
template int launch_add_increment<float>(const GridDev&, const float*, double*, float*, float*, float*, const Ctrl*, cudaStream_t);

}  // namespace dtt

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
// c_j = cos q_j), zeroing null modes (a_c <= threshold).
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
             int comp0, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
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

template <typename T>
int launch_transform_axis(const GridDev& g, const T* in, T* out, const TransformTables& tt,
                          int axis, int inverse, int ncomp_first, int ncomp, const Ctrl* ctrl,
                          cudaStream_t s) {
  const T* M[3];
  for (int c = 0; c < 3; ++c)
    M[c] = (const T*)(inverse ? tt.inv[c][axis] : tt.fwd[c][axis]);
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];
  if (axis == 0) {
    int rows = nny * nnz;
    dim3 grd((nnx + GBN - 1) / GBN, (rows + GBM - 1) / GBM, ncomp);
    k_axis_right<T><<<grd, 256, 0, s>>>(in, out, M[0], M[1], M[2], nnx, rows, g.nnodes, ncomp_first, ctrl);
  } else {
    int len = axis == 1 ? nny : nnz;
    int inner = axis == 1 ? nnx : nnx * nny;
    int outer = axis == 1 ? nnz : 1;
    dim3 grd((inner + GBN - 1) / GBN, (len + GBM - 1) / GBM, outer * ncomp);
    k_axis_left<T><<<grd, 256, 0, s>>>(in, out, M[0], M[1], M[2], len, inner, outer, g.nnodes, ncomp_first, ctrl);
  }
  return (int)cudaGetLastError();
}

template <typename T>
__global__ void k_green(const GridDev g, T* __restrict__ spec, const double* __restrict__ c0x,
                        const double* __restrict__ c0y, const double* __restrict__ c0z,
                        const double* __restrict__ c1x, const double* __restrict__ c1y,
                        const double* __restrict__ c1z, const double* __restrict__ c2x,
                        const double* __restrict__ c2y, const double* __restrict__ c2z, double lam0,
                        double mu0, double thr0, double thr1, double thr2, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  const long long NN = g.nnodes;
  const long long total = 3 * NN;
  const double ih2 = 1.0 / (g.h * g.h);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int c = (int)(e / NN);
    long long n = e - c * NN;
    int i = (int)(n % g.nn[0]);
    long long r = n / g.nn[0];
    int j = (int)(r % g.nn[1]);
    int k = (int)(r / g.nn[1]);
    const double* cx = c == 0 ? c0x : (c == 1 ? c1x : c2x);
    const double* cy = c == 0 ? c0y : (c == 1 ? c1y : c2y);
    const double* cz = c == 0 ? c0z : (c == 1 ? c1z : c2z);
    double X = cx[i], Y = cy[j], Z = cz[k];
    double Sx, Sy, Sz;
    if (g.scheme == SCHEME_TETRA2) {
      Sx = (1.0 + Y * Z - X * Y - X * Z) * ih2;
      Sy = (1.0 + X * Z - Y * X - Y * Z) * ih2;
      Sz = (1.0 + X * Y - Z * X - Z * Y) * ih2;
    } else {
      Sx = (1.0 - X) * (1.0 + Y) * (1.0 + Z) * 0.5 * ih2;
      Sy = (1.0 - Y) * (1.0 + X) * (1.0 + Z) * 0.5 * ih2;
      Sz = (1.0 - Z) * (1.0 + X) * (1.0 + Y) * 0.5 * ih2;
    }
    double Sc = c == 0 ? Sx : (c == 1 ? Sy : Sz);
    double a = lam0 * Sc + 2.0 * mu0 * (Sx + Sy + Sz);
    double thr = c == 0 ? thr0 : (c == 1 ? thr1 : thr2);
    spec[e] = (a <= thr) ? (T)0 : (T)((double)spec[e] / a);
  }
}

template <typename T>
int launch_green_multiply(const GridDev& g, T* spec, const TransformTables& tt, int scheme,
                          const Ctrl* ctrl, cudaStream_t s) {
  (void)scheme;
  long long total = 3 * g.nnodes;
  int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
  k_green<T><<<blocks, 256, 0, s>>>(g, spec, tt.cosq[0][0], tt.cosq[0][1], tt.cosq[0][2], tt.cosq[1][0],
                                    tt.cosq[1][1], tt.cosq[1][2], tt.cosq[2][0], tt.cosq[2][1],
                                    tt.cosq[2][2], tt.lam0, tt.mu0, tt.null_thr[0], tt.null_thr[1],
                                    tt.null_thr[2], ctrl);
  return (int)cudaGetLastError();
}

// u~ <- u~ + delta (Green step in increment form: G(p~) = u~ + G(p~ - A0 u~)).
template <typename T>
__global__ void k_add_increment(long long total, const T* __restrict__ delta, double* __restrict__ u64,
                                float* __restrict__ uhi, float* __restrict__ ulo, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
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
                         const Ctrl* ctrl, cudaStream_t s) {
  long long total = 3 * g.nnodes;
  int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
  k_add_increment<T><<<blocks, 256, 0, s>>>(total, delta, u64, uhi, ulo, ctrl);
  return (int)cudaGetLastError();
}

template int launch_transform_axis<double>(const GridDev&, const double*, double*, const TransformTables&, int, int, int, int, const Ctrl*, cudaStream_t);
template int launch_transform_axis<float>(const GridDev&, const float*, float*, const TransformTables&, int, int, int, int, const Ctrl*, cudaStream_t);
template int launch_green_multiply<double>(const GridDev&, double*, const TransformTables&, int, const Ctrl*, cudaStream_t);
template int launch_green_multiply<float>(const GridDev&, float*, const TransformTables&, int, const Ctrl*, cudaStream_t);
template int launch_add_increment<double>(const GridDev&, const double*, double*, float*, float*, const Ctrl*, cudaStream_t);
template int launch_add_increment<float>(const GridDev&, const float*, double*, float*, float*, const Ctrl*, cudaStream_t);

}  // namespace dtt

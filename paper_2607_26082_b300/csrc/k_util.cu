// Small utility kernels: precision conversion, float-float split/join, the stress output
// at the integration points (Section 3.1.1 gradients, sigma = lambda tr(eps) 1 + 2 mu eps,
// or the finite-strain stresses of Section 5.2) used by dtt_get_fields and
// dtt_get_stress_tensor, and the smallest det F over the integration points.  Not on the
// iteration path.
#include <algorithm>

#include "dtt_internal.cuh"

namespace dtt {

template <typename A, typename B>
__global__ void k_convert(long long n, const A* __restrict__ in, B* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (B)in[e];
}

__global__ void k_split(long long n, const double* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    float h, l;
    ff_set(h, l, in[e]);
    hi[e] = h;
    lo[e] = l;
  }
}

__global__ void k_join(long long n, const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)hi[e] + (double)lo[e];
}

static int nblk(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 16); }

int launch_to_double(long long n, const void* in, int in_is_float, double* out, cudaStream_t s) {
  if (in_is_float) k_convert<float, double><<<nblk(n), 256, 0, s>>>(n, (const float*)in, out);
  else k_convert<double, double><<<nblk(n), 256, 0, s>>>(n, (const double*)in, out);
  return (int)cudaGetLastError();
}
int launch_from_double(long long n, const double* in, void* out, int out_is_float, cudaStream_t s) {
  if (out_is_float) k_convert<double, float><<<nblk(n), 256, 0, s>>>(n, in, (float*)out);
  else k_convert<double, double><<<nblk(n), 256, 0, s>>>(n, in, (double*)out);
  return (int)cudaGetLastError();
}
// u~ = 0 on every Dirichlet-face DOF (a node on a face whose condition for the component
// is Dirichlet, periodic axes excepted): the DOFs the discrete problem removes
// Zeroes the Dirichlet DOFs: blockIdx.y = axis d and face f (2 d + f), blockIdx.z = component;
// the CTAs of a face sweep its node plane.
__global__ void k_zero_dirichlet(GridDev g, double* u64, float* uhi, float* ulo) {
  const int d = blockIdx.y >> 1, f = blockIdx.y & 1, c = blockIdx.z;
  if (g.periodic[d] || g.bc[d][f][c] != BC_D) return;
  const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;   // the plane's two axes
  const int n1 = g.nn[a1], n2 = g.nn[a2];
  const long long st[3] = {1, g.nn[0], (long long)g.nn[0] * g.nn[1]};
  const long long off = (long long)c * g.nnodes + (f ? (long long)(g.nn[d] - 1) * st[d] : 0);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n1 * n2; q += gridDim.x * blockDim.x) {
    const int i2 = q / n1, i1 = q - i2 * n1;
    const long long e = off + i1 * st[a1] + i2 * st[a2];
    if (u64) u64[e] = 0.0;
    if (uhi) uhi[e] = 0.f;
    if (ulo) ulo[e] = 0.f;
  }
}

int launch_zero_dirichlet(const GridDev& g, double* u64, float* uhi, float* ulo, cudaStream_t s) {
  int plane = 1;
  for (int d = 0; d < 3; ++d)
    for (int e = d + 1; e < 3; ++e) plane = std::max(plane, g.nn[d] * g.nn[e]);
  const int blocks = std::min((plane + 255) / 256, 148 * 4);
  k_zero_dirichlet<<<dim3(blocks, 6, 3), 256, 0, s>>>(g, u64, uhi, ulo);
  return (int)cudaGetLastError();
}

int launch_split(long long n, const double* in, float* hi, float* lo, cudaStream_t s) {
  k_split<<<nblk(n), 256, 0, s>>>(n, in, hi, lo);
  return (int)cudaGetLastError();
}
int launch_join(long long n, const float* hi, const float* lo, double* out, cudaStream_t s) {
  k_join<<<nblk(n), 256, 0, s>>>(n, hi, lo, out);
  return (int)cudaGetLastError();
}

// Stress at every integration point from a float64 u~ (3 x nnodes).  full = 0: the
// symmetric tensor, 6 values (xx yy zz yz xz xy) -- sigma in small strain, the second
// Piola-Kirchhoff S in finite strain; full = 1: the tensor paired with grad u, 9 values
// row c, column d -- sigma, or the first Piola-Kirchhoff Pi = F.S (Section 5.2).
struct Eps9 { double e[3][3]; };

// Displacement gradients G[t][c][d] = d u_c / d x_d at the integration points of voxel v
// (x fastest): TETRA2 two points (even / odd parity corners, 1 / 2h), HEX1 one (1 / 4h).
__device__ void voxel_gradients(const GridDev& g, const double* __restrict__ u, long long v, double G[2][3][3]) {
  int vx = (int)(v % g.nvox[0]);
  long long r = v / g.nvox[0];
  int vy = (int)(r % g.nvox[1]);
  int vz = (int)(r / g.nvox[1]);
  const int nip = g.scheme == SCHEME_TETRA2 ? 2 : 1;
  for (int t = 0; t < 2; ++t)
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) G[t][c][d] = 0.0;
  for (int q = 0; q < 8; ++q) {
    int dx = q & 1, dy = (q >> 1) & 1, dz = (q >> 2) & 1;
    int i = (vx + dx) % g.nn[0], j = (vy + dy) % g.nn[1], k = (vz + dz) % g.nn[2];
    long long n = i + (long long)g.nn[0] * (j + (long long)g.nn[1] * k);
    const int t = nip == 2 ? ((dx + dy + dz) & 1) : 0;
    const double coef = nip == 2 ? 1.0 / (2.0 * g.h) : 1.0 / (4.0 * g.h);
    const double s[3] = {dx ? 1.0 : -1.0, dy ? 1.0 : -1.0, dz ? 1.0 : -1.0};
    for (int c = 0; c < 3; ++c) {
      const double uc = u[(long long)c * g.nnodes + n];
      for (int d = 0; d < 3; ++d) G[t][c][d] += coef * s[d] * uc;
    }
  }
}

__global__ void k_stress_out(const GridDev g, const double* __restrict__ u, const uint8_t* __restrict__ phase,
                             const double* __restrict__ lam, const double* __restrict__ mu, const Eps9 eps, int full,
                             double* __restrict__ out) {
  const long long NV = (long long)g.nvox[0] * g.nvox[1] * g.nvox[2];
  const int nip = g.scheme == SCHEME_TETRA2 ? 2 : 1;
  const int nout = full ? 9 : 6;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < NV; v += (long long)gridDim.x * blockDim.x) {
    double GG[2][3][3];
    voxel_gradients(g, u, v, GG);
    double L = lam[phase[v]], M = mu[phase[v]];
    for (int t = 0; t < nip; ++t) {
      double (&G)[3][3] = GG[t];
      double H[3][3], E[3][3], S[3][3], P[3][3];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) H[c][d] = eps.e[c][d] + G[c][d];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
          double e = 0.5 * (H[p][q] + H[q][p]);
          if (g.finite_strain)
            for (int k = 0; k < 3; ++k) e += 0.5 * H[k][p] * H[k][q];
          E[p][q] = e;
        }
      const double tr = E[0][0] + E[1][1] + E[2][2];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) S[p][q] = 2 * M * E[p][q] + (p == q ? L * tr : 0.0);
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          double x = S[c][d];
          if (g.finite_strain)
            for (int k = 0; k < 3; ++k) x += H[c][k] * S[k][d];
          P[c][d] = x;
        }
      double* o = out + (v * nip + t) * nout;
      if (full) {
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) o[3 * c + d] = P[c][d];
      } else {
        o[0] = S[0][0];
        o[1] = S[1][1];
        o[2] = S[2][2];
        o[3] = S[1][2];
        o[4] = S[0][2];
        o[5] = S[0][1];
      }
    }
  }
}

// Smallest det F, F = 1 + eps* + grad u~, over every integration point; one value per
// block (the host takes the minimum of the blocks).
__global__ void k_min_jacobian(const GridDev g, const double* __restrict__ u, const Eps9 eps,
                               double* __restrict__ block_min) {
  __shared__ double red[256];
  const long long NV = (long long)g.nvox[0] * g.nvox[1] * g.nvox[2];
  const int nip = g.scheme == SCHEME_TETRA2 ? 2 : 1;
  double m = 1.0e300;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < NV; v += (long long)gridDim.x * blockDim.x) {
    double GG[2][3][3];
    voxel_gradients(g, u, v, GG);
    for (int t = 0; t < nip; ++t) {
      double F[3][3];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) F[c][d] = (c == d ? 1.0 : 0.0) + eps.e[c][d] + GG[t][c][d];
      const double det = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                         F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
      m = fmin(m, det);
    }
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) block_min[blockIdx.x] = red[0];
}

int min_jacobian_blocks(const GridDev& g) { return nblk((long long)g.nvox[0] * g.nvox[1] * g.nvox[2]); }

int launch_min_jacobian(const GridDev& g, const double* u, const double eps[3][3], double* block_min,
                        cudaStream_t s) {
  Eps9 e;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) e.e[p][q] = eps[p][q];
  k_min_jacobian<<<min_jacobian_blocks(g), 256, 0, s>>>(g, u, e, block_min);
  return (int)cudaGetLastError();
}

int launch_stress_out(const GridDev& g, const double* u, const uint8_t* phase, const double* lam,
                      const double* mu, const double eps[3][3], int full, double* out, cudaStream_t s) {
  long long NV = (long long)g.nvox[0] * g.nvox[1] * g.nvox[2];
  Eps9 e;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) e.e[p][q] = eps[p][q];
  k_stress_out<<<nblk(NV), 256, 0, s>>>(g, u, phase, lam, mu, e, full, out);
  return (int)cudaGetLastError();
}

}  // namespace dtt

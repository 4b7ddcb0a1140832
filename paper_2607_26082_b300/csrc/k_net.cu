// Kernels of the warm-start network (include/dtt_net.h): 3x3x3 convolutions as implicit
// GEMMs on the BF16 tensor cores (warp-level mma.sync m16n8k16, FP32 accumulation), with
// channels-last activations [voxel][channel] and weights [tap][cout][cin] (forward, backward
// data reads the [tap][cin][cout] copy), plus the pooling, upsampling, loss, feature and
// Adam kernels around them.
//
//   forward:        y[v][o]  = b[o] + sum_tap sum_i W[tap][o][i] x[v + off(tap)][i]
//   backward data:  dx[v][i] = sum_tap sum_o W[tap][o][i] dz[v - off(tap)][o]
//   backward weight dW[tap][o][i] = sum_v dz[v][o] x[v + off(tap)][i],  db[o] = sum_v dz[v][o]
// (zero outside the grid; off(tap) = (dx, dy, dz), tap = 9 (dz+1) + 3 (dy+1) + (dx+1)).
#include <cuda_bf16.h>

#include "dtt_internal.cuh"
#include "net_internal.cuh"

namespace dtt {
namespace net {

namespace {

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct Vox {
  int x, y, z;
  bool ok;
};

__device__ __forceinline__ Vox vox_of(long long v, int nx, int ny, long long V) {
  Vox r;
  r.ok = v < V;
  if (!r.ok) v = 0;
  r.x = (int)(v % nx);
  const long long q = v / nx;
  r.y = (int)(q % ny);
  r.z = (int)(q / ny);
  return r;
}

// linear index of voxel p shifted by (dx, dy, dz), or -1 outside the grid
__device__ __forceinline__ long long shifted(const Vox& p, int dx, int dy, int dz, int nx, int ny, int nz) {
  const int x = p.x + dx, y = p.y + dy, z = p.z + dz;
  if (!p.ok || x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return -1;
  return ((long long)z * ny + y) * nx + x;
}

}  // namespace

// ---- forward: CTA of 4 warps = 64 voxels x COUT; each warp 16 voxels x COUT
template <int CIN, int COUT, int FLAGS>
__global__ void __launch_bounds__(128)
k_conv_fwd(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
           int nx, int ny, int nz, __nv_bfloat16* __restrict__ Y, float* __restrict__ Yf,
           const __nv_bfloat16* __restrict__ skip, __nv_bfloat16* __restrict__ Rout) {
  constexpr int NT = COUT / 8, KC = CIN / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const long long V = (long long)nx * ny * nz;
  const long long m0 = ((long long)blockIdx.x * 4 + warp) * 16;
  const Vox p0 = vox_of(m0 + g, nx, ny, V), p1 = vox_of(m0 + g + 8, nx, ny, V);
  float acc[NT][4];
  #pragma unroll
  for (int j = 0; j < NT; ++j)
    #pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const long long s0 = shifted(p0, dx, dy, dz, nx, ny, nz), s1 = shifted(p1, dx, dy, dz, nx, ny, nz);
    const uint32_t* r0 = s0 >= 0 ? (const uint32_t*)(X + s0 * CIN) : nullptr;
    const uint32_t* r1 = s1 >= 0 ? (const uint32_t*)(X + s1 * CIN) : nullptr;
    const uint32_t* wt = (const uint32_t*)(Wt + (size_t)tap * COUT * CIN);
    #pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      uint32_t a[4];
      a[0] = r0 ? r0[kc * 8 + t4] : 0u;
      a[1] = r1 ? r1[kc * 8 + t4] : 0u;
      a[2] = r0 ? r0[kc * 8 + 4 + t4] : 0u;
      a[3] = r1 ? r1[kc * 8 + 4 + t4] : 0u;
      #pragma unroll
      for (int j = 0; j < NT; ++j) {
        const uint32_t* wr = wt + (size_t)(j * 8 + g) * (CIN / 2);
        uint32_t b[2] = {wr[kc * 8 + t4], wr[kc * 8 + 4 + t4]};
        mma_bf16(acc[j], a, b);
      }
    }
  }
  #pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int col = j * 8 + 2 * t4;
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long row = m0 + g + 8 * h;
      if (row >= V) continue;
      float v0 = acc[j][2 * h] + bias[col], v1 = acc[j][2 * h + 1] + bias[col + 1];
      if (FLAGS & CF_RELU) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      const size_t e = (size_t)row * COUT + col;
      if (FLAGS & CF_SKIP) {
        *(uint32_t*)(Rout + e) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
        v0 += __bfloat162float(skip[e]);
        v1 += __bfloat162float(skip[e + 1]);
      }
      if (FLAGS & CF_F32) {
        Yf[e] = v0;
        Yf[e + 1] = v1;
      } else {
        *(uint32_t*)(Y + e) = pack2(__float2bfloat16(v0), __float2bfloat16(v1));
      }
    }
  }
}

// ---- backward data: dX[v][i] = sum_tap sum_o Wd[tap][i][o] dZ[v - off][o]  (fp32 out)
template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
k_conv_bwd_data(const __nv_bfloat16* __restrict__ dZ, const __nv_bfloat16* __restrict__ Wd, int nx, int ny, int nz,
                float* __restrict__ dX) {
  constexpr int NT = CIN / 8, KC = COUT / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const long long V = (long long)nx * ny * nz;
  const long long m0 = ((long long)blockIdx.x * 4 + warp) * 16;
  const Vox p0 = vox_of(m0 + g, nx, ny, V), p1 = vox_of(m0 + g + 8, nx, ny, V);
  float acc[NT][4];
  #pragma unroll
  for (int j = 0; j < NT; ++j)
    #pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const long long s0 = shifted(p0, -dx, -dy, -dz, nx, ny, nz), s1 = shifted(p1, -dx, -dy, -dz, nx, ny, nz);
    const uint32_t* r0 = s0 >= 0 ? (const uint32_t*)(dZ + s0 * COUT) : nullptr;
    const uint32_t* r1 = s1 >= 0 ? (const uint32_t*)(dZ + s1 * COUT) : nullptr;
    const uint32_t* wd = (const uint32_t*)(Wd + (size_t)tap * CIN * COUT);
    #pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      uint32_t a[4];
      a[0] = r0 ? r0[kc * 8 + t4] : 0u;
      a[1] = r1 ? r1[kc * 8 + t4] : 0u;
      a[2] = r0 ? r0[kc * 8 + 4 + t4] : 0u;
      a[3] = r1 ? r1[kc * 8 + 4 + t4] : 0u;
      #pragma unroll
      for (int j = 0; j < NT; ++j) {
        const uint32_t* wr = wd + (size_t)(j * 8 + g) * (COUT / 2);
        uint32_t b[2] = {wr[kc * 8 + t4], wr[kc * 8 + 4 + t4]};
        mma_bf16(acc[j], a, b);
      }
    }
  }
  #pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int col = j * 8 + 2 * t4;
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long row = m0 + g + 8 * h;
      if (row >= V) continue;
      dX[(size_t)row * CIN + col] = acc[j][2 * h];
      dX[(size_t)row * CIN + col + 1] = acc[j][2 * h + 1];
    }
  }
}

// ---- backward weight: dW[tap][o][i] += sum over a chunk of voxels of dZ[v][o] X[v + off][i]
// (grid: voxel chunks x 27 taps; the (m-tile, n-tile) pairs of the [COUT x CIN] block are
// shared out among the 4 warps; FP32 atomics combine the chunks)
template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
k_conv_bwd_weight(const __nv_bfloat16* __restrict__ dZ, const __nv_bfloat16* __restrict__ X, int nx, int ny, int nz,
                  int chunk, float* __restrict__ dW) {
  constexpr int MT = COUT / 16, NTL = CIN / 8, P = MT * NTL, PW = (P + 3) / 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const long long V = (long long)nx * ny * nz;
  const int tap = blockIdx.y;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const long long v0 = (long long)blockIdx.x * chunk;
  const long long v1 = min(v0 + (long long)chunk, V);
  const unsigned short* dz16 = (const unsigned short*)dZ;
  const unsigned short* x16 = (const unsigned short*)X;
  float acc[PW][4];
  #pragma unroll
  for (int q = 0; q < PW; ++q)
    #pragma unroll
    for (int r = 0; r < 4; ++r) acc[q][r] = 0.f;
  for (long long kb = v0; kb < v1; kb += 16) {
    // the four voxels of this thread's k positions: kb + 2 t4 + {0, 1, 8, 9}
    long long kv[4] = {kb + 2 * t4, kb + 2 * t4 + 1, kb + 2 * t4 + 8, kb + 2 * t4 + 9};
    long long src[4];
    bool in[4];
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      in[q] = kv[q] < v1;
      const Vox p = vox_of(in[q] ? kv[q] : 0, nx, ny, V);
      src[q] = in[q] ? shifted(p, dx, dy, dz, nx, ny, nz) : -1;
    }
    #pragma unroll
    for (int q = 0; q < PW; ++q) {
      const int pr = warp + 4 * q;
      if (pr >= P) break;
      const int mt = pr / NTL, nt = pr % NTL;
      const int o0 = mt * 16 + g, o1 = o0 + 8;
      auto dzv = [&](int kq, int o) -> unsigned {
        return in[kq] ? (unsigned)dz16[(size_t)kv[kq] * COUT + o] : 0u;
      };
      uint32_t a[4];
      a[0] = dzv(0, o0) | (dzv(1, o0) << 16);
      a[1] = dzv(0, o1) | (dzv(1, o1) << 16);
      a[2] = dzv(2, o0) | (dzv(3, o0) << 16);
      a[3] = dzv(2, o1) | (dzv(3, o1) << 16);
      const int ci = nt * 8 + g;
      auto xv = [&](int kq) -> unsigned { return src[kq] >= 0 ? (unsigned)x16[(size_t)src[kq] * CIN + ci] : 0u; };
      uint32_t b[2] = {xv(0) | (xv(1) << 16), xv(2) | (xv(3) << 16)};
      mma_bf16(acc[q], a, b);
    }
  }
  #pragma unroll
  for (int q = 0; q < PW; ++q) {
    const int pr = warp + 4 * q;
    if (pr >= P) break;
    const int mt = pr / NTL, nt = pr % NTL;
    const int o0 = mt * 16 + g, col = nt * 8 + 2 * t4;
    float* w = dW + (size_t)tap * COUT * CIN;
    atomicAdd(&w[(size_t)o0 * CIN + col], acc[q][0]);
    atomicAdd(&w[(size_t)o0 * CIN + col + 1], acc[q][1]);
    atomicAdd(&w[(size_t)(o0 + 8) * CIN + col], acc[q][2]);
    atomicAdd(&w[(size_t)(o0 + 8) * CIN + col + 1], acc[q][3]);
  }
}

// ---- bias gradient: db[o] += sum_v dZ[v][o] (block partial sums, FP32 atomics)
template <int COUT>
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dZ, long long V, float* __restrict__ db) {
  __shared__ float sh[COUT];
  for (int o = threadIdx.x; o < COUT; o += blockDim.x) sh[o] = 0.f;
  __syncthreads();
  const int o = threadIdx.x % COUT;
  const int lanes = blockDim.x / COUT;
  float s = 0.f;
  for (long long v = (long long)blockIdx.x * lanes + threadIdx.x / COUT; v < V; v += (long long)gridDim.x * lanes)
    s += __bfloat162float(dZ[(size_t)v * COUT + o]);
  atomicAdd(&sh[o], s);
  __syncthreads();
  for (int q = threadIdx.x; q < COUT; q += blockDim.x) atomicAdd(&db[q], sh[q]);
}

// ---- elementwise pieces

// dZ = G where the layer's ReLU output R is positive (all of G without a ReLU), in BF16
__global__ void k_relu_bwd(const float* __restrict__ G, const __nv_bfloat16* __restrict__ R, long long n,
                           __nv_bfloat16* __restrict__ dZ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const bool on = R == nullptr || __bfloat162float(R[i]) > 0.f;
    dZ[i] = __float2bfloat16(on ? G[i] : 0.f);
  }
}

__host__ __device__ __forceinline__ int half_up(int n) { return (n + 1) / 2; }

// coarse[V'][C] = mean of the fine voxels of each 2x2x2 block (partial blocks at odd edges)
__global__ void k_pool_fwd(const __nv_bfloat16* __restrict__ in, int nx, int ny, int nz, int C,
                           __nv_bfloat16* __restrict__ out) {
  const int cx = half_up(nx), cy = half_up(ny), cz = half_up(nz);
  const long long n = (long long)cx * cy * cz * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long cv = i / C;
    const int X = (int)(cv % cx), Y = (int)((cv / cx) % cy), Z = (int)(cv / ((long long)cx * cy));
    float s = 0.f;
    int cnt = 0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x >= nx || y >= ny || z >= nz) continue;
          s += __bfloat162float(in[(((long long)z * ny + y) * nx + x) * C + c]);
          ++cnt;
        }
    out[i] = __float2bfloat16(s / (float)cnt);
  }
}

// gf[v][c] += gc[parent(v)][c] / (children of the parent)   (adjoint of k_pool_fwd)
__global__ void k_pool_bwd_add(const float* __restrict__ gc, int nx, int ny, int nz, int C, float* __restrict__ gf) {
  const int cx = half_up(nx), cy = half_up(ny);
  const long long n = (long long)nx * ny * nz * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    const int X = x / 2, Y = y / 2, Z = z / 2;
    const int cnt = (2 * X + 1 < nx ? 2 : 1) * (2 * Y + 1 < ny ? 2 : 1) * (2 * Z + 1 < nz ? 2 : 1);
    gf[i] += gc[(((long long)Z * cy + Y) * cx + X) * C + c] / (float)cnt;
  }
}

// fine[v][c] = coarse[parent(v)][c]
__global__ void k_up_fwd(const __nv_bfloat16* __restrict__ coarse, int nx, int ny, int nz, int C,
                         __nv_bfloat16* __restrict__ fine) {
  const int cx = half_up(nx), cy = half_up(ny);
  const long long n = (long long)nx * ny * nz * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    fine[i] = coarse[(((long long)(z / 2) * cy + y / 2) * cx + x / 2) * C + c];
  }
}

// gc[V'][c] = sum over the fine children (adjoint of k_up_fwd)
__global__ void k_up_bwd(const float* __restrict__ gf, int nx, int ny, int nz, int C, float* __restrict__ gc) {
  const int cx = half_up(nx), cy = half_up(ny), cz = half_up(nz);
  const long long n = (long long)cx * cy * cz * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long cv = i / C;
    const int X = (int)(cv % cx), Y = (int)((cv / cx) % cy), Z = (int)(cv / ((long long)cx * cy));
    float s = 0.f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x >= nx || y >= ny || z >= nz) continue;
          s += gf[(((long long)z * ny + y) * nx + x) * C + c];
        }
    gc[i] = s;
  }
}

__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] += b[i];
}

__global__ void k_f2bf(const float* __restrict__ a, long long n, __nv_bfloat16* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// loss = mean over nodes and channels 0..2 of d^2 + s2 * sum_axis (forward difference of d)^2,
// d = y - t (differences between neighbouring nodes inside the grid); gy = dloss/dy (0 on
// channels >= 3)
__device__ __forceinline__ float ddiff(const float* y, const float* t, long long v, int c, int CY) {
  return y[v * CY + c] - t[v * 3 + c];
}

__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, int nx, int ny, int nz, int CY,
                       float s2, float* __restrict__ gy, double* __restrict__ loss) {
  __shared__ double sh[8];
  const long long V = (long long)nx * ny * nz;
  double acc = 0.0;
  const float inv = 1.f / (3.f * (float)V);
  const long long st[3] = {1, nx, (long long)nx * ny};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * CY; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % CY);
    const long long v = i / CY;
    float gv = 0.f;
    if (c < 3) {
      const int idx[3] = {(int)(v % nx), (int)((v / nx) % ny), (int)(v / ((long long)nx * ny))};
      const int n[3] = {nx, ny, nz};
      const float d = ddiff(y, t, v, c, CY);
      float l = d * d, g = d;
      for (int a = 0; a < 3; ++a) {
        if (idx[a] + 1 < n[a]) {
          const float f = ddiff(y, t, v + st[a], c, CY) - d;
          l += s2 * f * f;
          g -= s2 * f;
        }
        if (idx[a] > 0) g += s2 * (d - ddiff(y, t, v - st[a], c, CY));
      }
      gv = 2.f * g * inv;
      acc += (double)l * (double)inv;
    }
    gy[i] = gv;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += sh[w];
    atomicAdd(loss, sum);
  }
}

// Adam on the FP32 master parameters; b1t, b2t = 1 - beta^t; the gradient is gscale * g
// (gscale = 1: the gradient as stored; 1/W: the mean of W ranks' summed gradients)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float b1t, float b2t, float eps, float gscale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / b1t) / (sqrtf(vi / b2t) + eps);
  }
}

// BF16 weight copies of one layer: Wt[tap][o][i] (forward) and Wd[tap][i][o] (backward data)
__global__ void k_relayout(const float* __restrict__ W, int cin, int cout, __nv_bfloat16* __restrict__ Wt,
                           __nv_bfloat16* __restrict__ Wd) {
  const long long n = 27LL * cin * cout;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % cin);
    const int o = (int)((q / cin) % cout);
    const int tap = (int)(q / ((long long)cin * cout));
    const __nv_bfloat16 b = __float2bfloat16(W[q]);
    Wt[q] = b;
    Wd[((long long)tap * cin + i) * cout + o] = b;
  }
}

// ---- launchers

namespace {
int grid_1d(long long n) {
  long long b = (n + 255) / 256;
  if (b > 148LL * 32) b = 148LL * 32;
  return (int)(b < 1 ? 1 : b);
}

template <int CIN, int COUT>
int conv_fwd_t(const ConvArgs& a, cudaStream_t s) {
  const long long V = (long long)a.nx * a.ny * a.nz;
  const unsigned blocks = (unsigned)((V + 63) / 64);
  switch (a.flags) {
    case CF_RELU:
      k_conv_fwd<CIN, COUT, CF_RELU><<<blocks, 128, 0, s>>>(a.x, a.wt, a.bias, a.nx, a.ny, a.nz, a.y, a.yf, a.skip, a.r);
      break;
    case CF_RELU | CF_SKIP:
      k_conv_fwd<CIN, COUT, CF_RELU | CF_SKIP><<<blocks, 128, 0, s>>>(a.x, a.wt, a.bias, a.nx, a.ny, a.nz, a.y, a.yf,
                                                                     a.skip, a.r);
      break;
    case CF_F32:
      k_conv_fwd<CIN, COUT, CF_F32><<<blocks, 128, 0, s>>>(a.x, a.wt, a.bias, a.nx, a.ny, a.nz, a.y, a.yf, a.skip, a.r);
      break;
    default:
      return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <int CIN, int COUT>
int conv_bwd_t(const ConvArgs& a, cudaStream_t s) {
  const long long V = (long long)a.nx * a.ny * a.nz;
  if (a.dx) {
    k_conv_bwd_data<CIN, COUT><<<(unsigned)((V + 63) / 64), 128, 0, s>>>(a.dz, a.wd, a.nx, a.ny, a.nz, a.dx);
    if (cudaError_t e = cudaGetLastError()) return (int)e;
  }
  const int chunk = 2048;
  dim3 grd((unsigned)((V + chunk - 1) / chunk), 27);
  k_conv_bwd_weight<CIN, COUT><<<grd, 128, 0, s>>>(a.dz, a.x, a.nx, a.ny, a.nz, chunk, a.dw);
  if (cudaError_t e = cudaGetLastError()) return (int)e;
  k_bias_grad<COUT><<<grid_1d(V * COUT / 8), 256, 0, s>>>(a.dz, V, a.db);
  return (int)cudaGetLastError();
}

template <int CIN>
int conv_fwd_c(const ConvArgs& a, cudaStream_t s) {
  switch (a.cout) {
    case 16: return conv_fwd_t<CIN, 16>(a, s);
    case 32: return conv_fwd_t<CIN, 32>(a, s);
    case 64: return conv_fwd_t<CIN, 64>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
template <int CIN>
int conv_bwd_c(const ConvArgs& a, cudaStream_t s) {
  switch (a.cout) {
    case 16: return conv_bwd_t<CIN, 16>(a, s);
    case 32: return conv_bwd_t<CIN, 32>(a, s);
    case 64: return conv_bwd_t<CIN, 64>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
}  // namespace

int launch_conv_fwd(const ConvArgs& a, cudaStream_t s) {
  switch (a.cin) {
    case 16: return conv_fwd_c<16>(a, s);
    case 32: return conv_fwd_c<32>(a, s);
    case 64: return conv_fwd_c<64>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_conv_bwd(const ConvArgs& a, cudaStream_t s) {
  switch (a.cin) {
    case 16: return conv_bwd_c<16>(a, s);
    case 32: return conv_bwd_c<32>(a, s);
    case 64: return conv_bwd_c<64>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_relu_bwd(const float* G, const __nv_bfloat16* R, long long n, __nv_bfloat16* dZ, cudaStream_t s) {
  k_relu_bwd<<<grid_1d(n), 256, 0, s>>>(G, R, n, dZ);
  return (int)cudaGetLastError();
}
int launch_pool_fwd(const __nv_bfloat16* in, int nx, int ny, int nz, int C, __nv_bfloat16* out, cudaStream_t s) {
  k_pool_fwd<<<grid_1d((long long)half_up(nx) * half_up(ny) * half_up(nz) * C), 256, 0, s>>>(in, nx, ny, nz, C, out);
  return (int)cudaGetLastError();
}
int launch_pool_bwd_add(const float* gc, int nx, int ny, int nz, int C, float* gf, cudaStream_t s) {
  k_pool_bwd_add<<<grid_1d((long long)nx * ny * nz * C), 256, 0, s>>>(gc, nx, ny, nz, C, gf);
  return (int)cudaGetLastError();
}
int launch_up_fwd(const __nv_bfloat16* coarse, int nx, int ny, int nz, int C, __nv_bfloat16* fine, cudaStream_t s) {
  k_up_fwd<<<grid_1d((long long)nx * ny * nz * C), 256, 0, s>>>(coarse, nx, ny, nz, C, fine);
  return (int)cudaGetLastError();
}
int launch_up_bwd(const float* gf, int nx, int ny, int nz, int C, float* gc, cudaStream_t s) {
  k_up_bwd<<<grid_1d((long long)half_up(nx) * half_up(ny) * half_up(nz) * C), 256, 0, s>>>(gf, nx, ny, nz, C, gc);
  return (int)cudaGetLastError();
}
int launch_add(float* a, const float* b, long long n, cudaStream_t s) {
  k_add<<<grid_1d(n), 256, 0, s>>>(a, b, n);
  return (int)cudaGetLastError();
}
int launch_f2bf(const float* a, long long n, __nv_bfloat16* b, cudaStream_t s) {
  k_f2bf<<<grid_1d(n), 256, 0, s>>>(a, n, b);
  return (int)cudaGetLastError();
}
int launch_loss(const float* y, const float* t, int nx, int ny, int nz, int CY, float s2, float* gy, double* loss,
                cudaStream_t s) {
  k_loss<<<grid_1d((long long)nx * ny * nz * CY), 256, 0, s>>>(y, t, nx, ny, nz, CY, s2, gy, loss);
  return (int)cudaGetLastError();
}
int launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s,
                float gscale) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float b1t = 1.f - powf(b1, (float)step), b2t = 1.f - powf(b2, (float)step);
  k_adam<<<grid_1d(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, b1t, b2t, 1e-8f, gscale);
  return (int)cudaGetLastError();
}
int launch_relayout(const float* W, int cin, int cout, __nv_bfloat16* Wt, __nv_bfloat16* Wd, cudaStream_t s) {
  k_relayout<<<grid_1d(27LL * cin * cout), 256, 0, s>>>(W, cin, cout, Wt, Wd);
  return (int)cudaGetLastError();
}

// ---- input features of a grid's nodes (layout in include/dtt_net.h)
__global__ void k_features(FeatArgs a) {
  const GridDev& g = a.g;
  const long long n = win_volume(a.w);
  for (long long vw = blockIdx.x * (long long)blockDim.x + threadIdx.x; vw < n; vw += (long long)gridDim.x * blockDim.x) {
    const int idx[3] = {a.w.o[0] + (int)(vw % a.w.n[0]), a.w.o[1] + (int)((vw / a.w.n[0]) % a.w.n[1]),
                        a.w.o[2] + (int)(vw / ((long long)a.w.n[0] * a.w.n[1]))};
    const long long v = idx[0] + (long long)g.nn[0] * (idx[1] + (long long)g.nn[1] * idx[2]);
    float es = 0.f;
    int cnt = 0;
    for (int oz = -1; oz <= 0; ++oz)
      for (int oy = -1; oy <= 0; ++oy)
        for (int ox = -1; ox <= 0; ++ox) {
          const int o[3] = {ox, oy, oz};
          int w[3];
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            int q = idx[d] + o[d];
            if (g.periodic[d]) q = (q + g.nvox[d]) % g.nvox[d];
            else if (q < 0 || q >= g.nvox[d]) ok = false;
            w[d] = q;
          }
          if (!ok) continue;
          es += a.enorm[a.phase[w[0] + (long long)g.nvox[0] * (w[1] + (long long)g.nvox[1] * w[2])]];
          ++cnt;
        }
    float* x = a.x + vw * 16;
    x[0] = cnt ? es / (float)cnt : 0.f;
    const uint8_t cm = a.cmask ? a.cmask[v] : 0;
    for (int c = 0; c < 3; ++c) {
      bool fixed = (cm >> c) & 1;
      for (int d = 0; d < 3; ++d) {
        if (g.periodic[d]) continue;
        if (idx[d] == 0 && g.bc[d][0][c] == BC_D) fixed = true;
        if (idx[d] == g.nn[d] - 1 && g.bc[d][1][c] == BC_D) fixed = true;
      }
      x[1 + c] = fixed ? 1.f : 0.f;
    }
    for (int q = 0; q < 6; ++q) x[4 + q] = a.eps6[q];
    for (int d = 0; d < 3; ++d) x[10 + d] = (float)idx[d] / (float)g.nvox[d];
    x[13] = x[14] = x[15] = 0.f;
  }
}

int launch_features(const FeatArgs& a, cudaStream_t s) {
  k_features<<<grid_1d(win_volume(a.w)), 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}

// ---- increment mode ---------------------------------------------------------------------
__device__ __forceinline__ double inc_u1(const IncArgs& a, long long i) {
  return a.u64 ? a.u64[i] : (double)a.uhi[i] + (double)a.ulo[i];
}

// fmax = max over the surface of -fn_prev (the previous increment's largest contact
// pressure): non-negative floats order like their bit patterns
__global__ void k_inc_fmax(IncArgs a) {
  float m = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.nface; q += gridDim.x * blockDim.x)
    m = fmaxf(m, (float)(-inc_fn(a, q)));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax((int*)a.fmax, __float_as_int(m));
}

__device__ __forceinline__ long long win_to_grid(const IncArgs& a, long long vw) {
  const int i = a.w.o[0] + (int)(vw % a.w.n[0]), j = a.w.o[1] + (int)((vw / a.w.n[0]) % a.w.n[1]),
            k = a.w.o[2] + (int)(vw / ((long long)a.w.n[0] * a.w.n[1]));
  return i + (long long)a.g.nn[0] * (j + (long long)a.g.nn[1] * k);
}
// window index of grid node n, or -1 outside the window
__device__ __forceinline__ long long grid_to_win(const IncArgs& a, long long n) {
  int idx[3] = {(int)(n % a.g.nn[0]), (int)((n / a.g.nn[0]) % a.g.nn[1]), (int)(n / ((long long)a.g.nn[0] * a.g.nn[1]))};
  for (int d = 0; d < 3; ++d) {
    idx[d] -= a.w.o[d];
    if (idx[d] < 0 || idx[d] >= a.w.n[d]) return -1;
  }
  return idx[0] + (long long)a.w.n[0] * (idx[1] + (long long)a.w.n[1] * idx[2]);
}
// the secant prediction of u~ at DOF i, divided by dd
__device__ __forceinline__ double inc_secant(const IncArgs& a, long long i) {
  return (inc_u1(a, i) - (a.u2 ? a.u2[i] : 0.0)) * a.s_sec / a.dd;
}

// channels 4-6: the secant prediction of the increment divided by dd; 7-9 cleared
__global__ void k_inc_nodes(IncArgs a) {
  const long long V = a.g.nnodes, Vw = win_volume(a.w);
  for (long long vw = blockIdx.x * (long long)blockDim.x + threadIdx.x; vw < Vw; vw += (long long)gridDim.x * blockDim.x) {
    const long long v = win_to_grid(a, vw);
    float* x = a.x + vw * 16;
    for (int c = 0; c < 3; ++c) x[4 + c] = (float)inc_secant(a, c * V + v);
    x[7] = x[8] = x[9] = 0.f;
  }
}

// surface nodes in the window: channel 7 = 1, 8 = gap of the secant-predicted position to
// the moved sphere over dd (clipped to +-8), 9 = previous pressure over its maximum
__global__ void k_inc_surface(IncArgs a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nface) return;
  const long long V = a.g.nnodes;
  const long long n = a.node[q];
  const long long vw = grid_to_win(a, n);
  if (vw < 0) return;
  const int idx[3] = {(int)(n % a.g.nn[0]), (int)((n / a.g.nn[0]) % a.g.nn[1]), (int)(n / ((long long)a.g.nn[0] * a.g.nn[1]))};
  float* x = a.x + vw * 16;
  double X[3], r2 = 0.0;
  for (int c = 0; c < 3; ++c) X[c] = a.g.h * idx[c];
  for (int c = 0; c < 3; ++c) {
    const double us = a.eps[c][0] * X[0] + a.eps[c][1] * X[1] + a.eps[c][2] * X[2];
    const double m = X[c] + us + inc_u1(a, c * V + n) + a.dd * inc_secant(a, c * V + n);
    r2 += (m - a.center[c]) * (m - a.center[c]);
  }
  const double gap = sqrt(r2) - a.radius;
  const float fm = *a.fmax;
  x[7] = 1.f;
  x[8] = fminf(8.f, fmaxf(-8.f, (float)(gap / a.dd)));
  x[9] = fm > 0.f ? (float)(-inc_fn(a, q)) / fm : 0.f;
}

__global__ void k_inc_targets(IncArgs a, const double* __restrict__ ut, float* __restrict__ t,
                              float* __restrict__ m) {
  const long long V = a.g.nnodes, Vw = win_volume(a.w);
  for (long long vw = blockIdx.x * (long long)blockDim.x + threadIdx.x; vw < Vw; vw += (long long)gridDim.x * blockDim.x) {
    const long long v = win_to_grid(a, vw);
    for (int c = 0; c < 3; ++c) {
      const long long i = c * V + v;
      // clipped: a node whose contact state flips can carry a correction far above the
      // others' (|t| <= 0.4 elsewhere on the training seeds)
      const double ti = (ut[i] - inc_u1(a, i)) / a.dd - inc_secant(a, i);
      t[vw * 4 + c] = (float)fmin(8.0, fmax(-8.0, ti));
    }
    t[vw * 4 + 3] = 0.f;
    m[vw] = 0.f;
  }
}
__global__ void k_inc_targets_surface(IncArgs a, const double* __restrict__ fnt, float* __restrict__ t,
                                      float* __restrict__ m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nface) return;
  const long long vw = grid_to_win(a, a.node[q]);
  if (vw < 0) return;
  const float fm = *a.fmax;
  // pressure over the previous increment's largest, clipped to [0, 4] (it grows by a few
  // per cent per increment; a spike at one node would otherwise dominate the loss)
  t[vw * 4 + 3] = fm > 0.f ? fminf(4.f, fmaxf(0.f, (float)(-fnt[q]) / fm)) : 0.f;
  m[vw] = 1.f;
}

// loss = mean over window nodes and the three displacement channels of (y - t)^2 + wp *
// mean over the window's surface nodes of (y3 - t3)^2; gy = dloss/dy
__global__ void k_inc_loss(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ m,
                           long long V, int CY, float inv3v, float wp_ns, float* __restrict__ gy,
                           double* __restrict__ loss) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * CY; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % CY);
    const long long v = i / CY;
    float g = 0.f;
    if (c < 3) {
      const float d = y[i] - t[v * 4 + c];
      acc += (double)(d * d) * inv3v;
      g = 2.f * d * inv3v;
    } else if (c == 3 && m[v] != 0.f) {
      const float d = y[i] - t[v * 4 + 3];
      acc += (double)(d * d) * wp_ns;
      g = 2.f * d * wp_ns;
    }
    gy[i] = g;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    atomicAdd(loss, s);
  }
}

// Weight of the correction at a window node: 1 inside, falling linearly to 0 over the last
// WIN_TAPER nodes before each window face that lies inside the grid (the contact face and
// the grid's own faces keep 1), so that the guess has no jump where the correction ends.
constexpr int WIN_TAPER = 8;

// every node: u = u~_(k-1) + dd (secant + tapered correction), the correction 0 outside
// the window
// One CTA per node row (c, z, y), threads along x: the window test and the taper of the row
// are fixed once, the secant factor s / dd comes from the host (no FP64 division and no
// 64-bit index division per value).
__global__ void k_inc_guess(IncArgs a, const float* __restrict__ y, int CY, double sec, double* __restrict__ u) {
  const int nx = a.g.nn[0], ny = a.g.nn[1], nz = a.g.nn[2];
  const int rows = 3 * ny * nz;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int c = r / (ny * nz), rz = r - c * ny * nz, zz = rz / ny, yy = rz - zz * ny;
    const long long base = (long long)c * a.g.nnodes + ((long long)zz * ny + yy) * nx;
    const int wy = yy - a.w.o[1], wz = zz - a.w.o[2];
    const bool rin = wy >= 0 && wy < a.w.n[1] && wz >= 0 && wz < a.w.n[2];
    double trow = 1.0;   // taper along y and z
    if (rin) {
      const int idx[3] = {0, wy, wz};
      for (int d = 1; d < 3; ++d) {
        if (a.w.o[d] > 0) trow = fmin(trow, (idx[d] + 1) / (double)(WIN_TAPER + 1));
        if (a.w.o[d] + a.w.n[d] < a.g.nn[d]) trow = fmin(trow, (a.w.n[d] - idx[d]) / (double)(WIN_TAPER + 1));
      }
    }
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const long long i = base + x;
      const int wx = x - a.w.o[0];
      double corr = 0.0;
      if (rin && wx >= 0 && wx < a.w.n[0]) {
        double t = trow;
        if (a.w.o[0] > 0) t = fmin(t, (wx + 1) / (double)(WIN_TAPER + 1));
        if (a.w.o[0] + a.w.n[0] < nx) t = fmin(t, (a.w.n[0] - wx) / (double)(WIN_TAPER + 1));
        const long long vw = wx + (long long)a.w.n[0] * (wy + (long long)a.w.n[1] * wz);
        corr = t * (double)y[vw * CY + c];
      }
      const double u1 = inc_u1(a, i);
      u[i] = u1 + a.dd * ((u1 - (a.u2 ? a.u2[i] : 0.0)) * sec + corr);
    }
  }
}
// surface nodes: in the initial zone when they carried pressure at the previous increment
// (fn_prev < 0: under monotone loading the zone grows) or where the predicted pressure
// exceeds thr (inside the window)
__global__ void k_inc_active(IncArgs a, const float* __restrict__ y, int CY, float thr, uint8_t* __restrict__ act) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nface) return;
  const long long vw = grid_to_win(a, a.node[q]);
  act[q] = (inc_fn(a, q) < 0.0 || (vw >= 0 && y[vw * CY + 3] > thr)) ? 1 : 0;
}

int launch_inc_fmax(const IncArgs& a, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.fmax, 0, sizeof(float), s);
  if (e != cudaSuccess) return (int)e;
  if (a.nface > 0) k_inc_fmax<<<(a.nface + 255) / 256, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}
int launch_inc_features(const IncArgs& a, cudaStream_t s) {
  k_inc_nodes<<<grid_1d(win_volume(a.w)), 256, 0, s>>>(a);
  if (a.nface > 0) k_inc_surface<<<(a.nface + 255) / 256, 256, 0, s>>>(a);
  return (int)cudaGetLastError();
}
int launch_inc_targets(const IncArgs& a, const double* u_target, const double* fn_target, float* t, float* m,
                       cudaStream_t s) {
  k_inc_targets<<<grid_1d(win_volume(a.w)), 256, 0, s>>>(a, u_target, t, m);
  if (a.nface > 0) k_inc_targets_surface<<<(a.nface + 255) / 256, 256, 0, s>>>(a, fn_target, t, m);
  return (int)cudaGetLastError();
}
int launch_inc_loss(const float* y, const float* t, const float* m, long long V, int CY, float wp, float* gy,
                    double* loss, cudaStream_t s) {
  // the number of surface nodes enters through wp (wp / Ns computed by the caller)
  k_inc_loss<<<grid_1d(V * CY), 256, 0, s>>>(y, t, m, V, CY, 1.f / (3.f * (float)V), wp, gy, loss);
  return (int)cudaGetLastError();
}
int launch_inc_guess(const IncArgs& a, const float* y, int CY, float thr, double* u, uint8_t* active,
                     cudaStream_t s) {
  const int rows = 3 * a.g.nn[1] * a.g.nn[2];
  k_inc_guess<<<rows < 148 * 32 ? rows : 148 * 32, 128, 0, s>>>(a, y, CY, a.s_sec / a.dd, u);
  if (a.nface > 0 && active) k_inc_active<<<(a.nface + 255) / 256, 256, 0, s>>>(a, y, CY, thr, active);
  return (int)cudaGetLastError();
}

// u[c][v] = scale * y[v][c] for c < 3 (network output to a u~ guess, float64, grid layout)
__global__ void k_out_to_u(const float* __restrict__ y, long long V, int CY, double scale, double* __restrict__ u) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * V; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / V);
    const long long v = i - c * V;
    u[i] = scale * (double)y[v * CY + c];
  }
}

int launch_out_to_u(const float* y, long long V, int CY, double scale, double* u, cudaStream_t s) {
  k_out_to_u<<<grid_1d(3 * V), 256, 0, s>>>(y, V, CY, scale, u);
  return (int)cudaGetLastError();
}

}  // namespace net
}  // namespace dtt

// Stress / divergence / reference-operator kernel of the mixed path (same operator as
// k_residual.cu: Eq. 3 with the HEX1 / TETRA2 gradients of Section 3.1.1, the Paux
// reference medium of Section 3.2.3 and the symmetry weights W of Table 1), organised for
// FP32 throughput on B300:
//
//  * one thread per node, a 32 x 8 node tile per CTA marching along z;
//  * every node evaluates, for each of its 8 voxels, only the integration point whose
//    tetrahedron contains it (TETRA2) or the voxel's single point (HEX1) -- FP32 work is
//    cheap, and this removes the per-voxel shared-memory stage and two of its barriers;
//  * u~ (float-float hi / lo), the step Delta and the voxel phases of the planes k-1..k+2
//    sit in a 4-slot shared-memory ring filled with cp.async one plane ahead, so the
//    global loads of plane k+2 overlap the arithmetic of plane k (one barrier per plane);
//  * in the Anderson difference form the kernel also accumulates the Gram row
//    <R_{i-1}, R_k> (k = 0..3) over the unconstrained DOFs; the projection kernels add the
//    constrained ones after they have shifted R_{i-1}.
// Partial sums per CTA (FP64 across threads): [sum w sigma:sigma, sum p^2, Gram 0..3].
#include "dtt_internal.cuh"

namespace dtt {

constexpr int FTX = 32, FTY = 8, FNP = 4;
constexpr int FHX = FTX + 2, FHY = FTY + 2;
constexpr int FPLANE = 3 * FHY * FHX;   // floats per plane (3 components)

__device__ __forceinline__ void cp_async4(void* smem_ptr, const void* gptr) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gptr));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrapi(int i, int n, int per) {
  if (per) { i %= n; if (i < 0) i += n; return i; }
  return (i < 0 || i >= n) ? -1 : i;
}

struct F32Tile {
  const float* H;   // hi, base of the 4-plane ring
  const float* Lo;  // lo
  const float* D;   // Delta
};

// value accessors: plane slot, component, local y, local x
__device__ __forceinline__ int sidx(int slot, int c, int ly, int lx) { return ((slot * 3 + c) * FHY + ly) * FHX + lx; }

template <int SCHEME>
__global__ void __launch_bounds__(FTX * FTY)
k_residual_f32(ResidualArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sH = (float*)smem_raw;
  float* sL = sH + FNP * FPLANE;
  float* sD = sL + FNP * FPLANE;
  uint8_t* sP = (uint8_t*)(sD + FNP * FPLANE);   // [FNP][FHY][FHX] voxel phases
  __shared__ float sLam[MAX_PHASE], sMu[MAX_PHASE];
  __shared__ double sRed[6][FTX * FTY / 32];

  if (a.ctrl && a.ctrl->done) return;
  const GridDev& g = a.g;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FTX + tx;
  for (int q = tid; q < a.nphase; q += FTX * FTY) {
    sLam[q] = (float)a.lam[q];
    sMu[q] = (float)a.mu[q];
  }
  const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
  const int zc = a.zchunk;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, g.nn[2]);
  const long long NN = g.nnodes;
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];

  // outputs by mode
  float* po = (float*)a.pout;
  float* xo = nullptr;
  float* ro = nullptr;
  const float* gprev = nullptr;
  const float* dfield = nullptr;
  const float* Rk[4] = {nullptr, nullptr, nullptr, nullptr};
  int rslot = -1;
  bool tau_on = true, tau_from_delta = false;
  if (a.mode == 0) {
    xo = (float*)a.xout;
  } else if (a.mode == 1) {
    const int il = a.ctrl->i_local;
    po = (float*)a.pring[il % 4];
    if (il > 0) {
      rslot = (il - 1) % 4;
      ro = (float*)a.rring[rslot];
      gprev = (const float*)a.gring[rslot];
      dfield = (const float*)a.dfield;
      tau_from_delta = true;
      for (int q = 0; q < 4; ++q) Rk[q] = (const float*)a.rring[q];
    } else {
      tau_on = false;
    }
  } else {
    tau_on = false;
  }
  const float lam0 = (float)a.lam0, mu0 = (float)a.mu0;
  float eps[3][3];
  #pragma unroll
  for (int p = 0; p < 3; ++p)
    #pragma unroll
    for (int q = 0; q < 3; ++q) eps[p][q] = (float)a.eps[p][q];
  const float c4h = (float)(1.0 / (4.0 * g.h));
  const float inv2h = (float)(1.0 / (2.0 * g.h));
  const float inv4h = (float)(1.0 / (4.0 * g.h));

  // ---- plane loader: node plane kk into ring slot, voxel phase plane kk into ring slot
  auto load_plane = [&](int kk) {
    const int slot = (kk + 8) & (FNP - 1);
    const int kw = wrapi(kk, nnz, g.periodic[2]);
    for (int q = tid; q < FHX * FHY; q += FTX * FTY) {
      const int lx = q % FHX, ly = q / FHX;
      const int gi = wrapi(x0 - 1 + lx, nnx, g.periodic[0]);
      const int gj = wrapi(y0 - 1 + ly, nny, g.periodic[1]);
      const bool ok = kw >= 0 && gi >= 0 && gj >= 0;
      const long long n = ok ? gi + (long long)nnx * (gj + (long long)nny * kw) : 0;
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int si = sidx(slot, c, ly, lx);
        if (ok) {
          cp_async4(&sH[si], a.uhi + c * NN + n);
          cp_async4(&sL[si], a.ulo + c * NN + n);
          if (dfield) cp_async4(&sD[si], dfield + c * NN + n);
        } else {
          sH[si] = 0.f;
          sL[si] = 0.f;
          sD[si] = 0.f;
        }
      }
      // voxel (x0-1+lx, y0-1+ly, kk)
      const int vx = wrapi(x0 - 1 + lx, g.nvox[0], g.periodic[0]);
      const int vy = wrapi(y0 - 1 + ly, g.nvox[1], g.periodic[1]);
      const int vz = wrapi(kk, g.nvox[2], g.periodic[2]);
      uint8_t ph = 255;   // 255 = no voxel
      if (vx >= 0 && vy >= 0 && vz >= 0) ph = a.phase[vx + (long long)g.nvox[0] * (vy + (long long)g.nvox[1] * vz)];
      sP[(slot * FHY + ly) * FHX + lx] = ph;
    }
  };

  double acc_s2 = 0.0, acc_p2 = 0.0;
  double acc_g[4] = {0.0, 0.0, 0.0, 0.0};

  load_plane(z0 - 1);
  load_plane(z0);
  load_plane(z0 + 1);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  const int i = x0 + tx, j = y0 + ty;
  const bool active = (i < nnx && j < nny);
  for (int k = z0; k < z1; ++k) {
    load_plane(k + 2);
    cp_async_commit();
    if (active) {
      float Fs[3] = {0.f, 0.f, 0.f}, F0[3] = {0.f, 0.f, 0.f};
      float s2loc = 0.f;
      #pragma unroll
      for (int ez = 0; ez < 2; ++ez) {
        const int sl0 = (k - 1 + ez + 8) & (FNP - 1);   // lower node plane of the voxel
        const int sl1 = (k + ez + 8) & (FNP - 1);
        #pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
          #pragma unroll
          for (int ex = 0; ex < 2; ++ex) {
            const int lx = tx + ex, ly = ty + ey;   // voxel lower corner in tile coordinates
            const uint8_t ph = sP[(sl0 * FHY + ly) * FHX + lx];
            if (ph == 255) continue;
            const float lam = sLam[ph], mu = sMu[ph];
            // node is corner delta = (1-ex, 1-ey, 1-ez) of this voxel
            const int dx = 1 - ex, dy = 1 - ey, dz = 1 - ez;
            const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
            float G[3][3], GD[3][3];
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
              auto u = [&](int cx, int cy, int cz) -> float2 {
                const int si = sidx(cz ? sl1 : sl0, c, ly + cy, lx + cx);
                return make_float2(sH[si], sL[si]);
              };
              auto dd = [&](int cx, int cy, int cz) -> float {
                return sD[sidx(cz ? sl1 : sl0, c, ly + cy, lx + cx)];
              };
              auto df = [](float2 p, float2 q) -> float {
                return __fadd_rn(__fsub_rn(p.x, q.x), __fsub_rn(p.y, q.y));
              };
              if constexpr (SCHEME == SCHEME_TETRA2) {
                if (((dx + dy + dz) & 1) == 0) {
                  // T1 = {000, 110, 101, 011}
                  const float2 a0 = u(0, 0, 0), b0 = u(1, 1, 0), c0 = u(1, 0, 1), e0 = u(0, 1, 1);
                  const float d_ba = df(b0, a0), d_ce = df(c0, e0), d_ca = df(c0, a0), d_eb = df(e0, b0);
                  G[c][0] = (d_ba + d_ce) * inv2h;
                  G[c][1] = (d_ba - d_ce) * inv2h;
                  G[c][2] = (d_ca + d_eb) * inv2h;
                  if (tau_from_delta) {
                    const float A = dd(0, 0, 0), B = dd(1, 1, 0), Cc = dd(1, 0, 1), E = dd(0, 1, 1);
                    GD[c][0] = ((B - A) + (Cc - E)) * inv2h;
                    GD[c][1] = ((B - A) - (Cc - E)) * inv2h;
                    GD[c][2] = ((Cc - A) + (E - B)) * inv2h;
                  }
                } else {
                  // T2 = {100, 010, 001, 111}
                  const float2 a1 = u(1, 0, 0), b1 = u(0, 1, 0), c1 = u(0, 0, 1), e1 = u(1, 1, 1);
                  const float e_ab = df(a1, b1), e_ec = df(e1, c1), e_ca = df(c1, a1), e_eb = df(e1, b1);
                  G[c][0] = (e_ab + e_ec) * inv2h;
                  G[c][1] = (e_ec - e_ab) * inv2h;
                  G[c][2] = (e_ca + e_eb) * inv2h;
                  if (tau_from_delta) {
                    const float A = dd(1, 0, 0), B = dd(0, 1, 0), Cc = dd(0, 0, 1), E = dd(1, 1, 1);
                    GD[c][0] = ((A - B) + (E - Cc)) * inv2h;
                    GD[c][1] = ((E - Cc) - (A - B)) * inv2h;
                    GD[c][2] = ((Cc - A) + (E - B)) * inv2h;
                  }
                }
              } else {
                const float2 u000 = u(0, 0, 0), u100 = u(1, 0, 0), u010 = u(0, 1, 0), u110 = u(1, 1, 0);
                const float2 u001 = u(0, 0, 1), u101 = u(1, 0, 1), u011 = u(0, 1, 1), u111 = u(1, 1, 1);
                G[c][0] = (df(u100, u000) + df(u110, u010) + df(u101, u001) + df(u111, u011)) * inv4h;
                G[c][1] = (df(u010, u000) + df(u110, u100) + df(u011, u001) + df(u111, u101)) * inv4h;
                G[c][2] = (df(u001, u000) + df(u101, u100) + df(u011, u010) + df(u111, u110)) * inv4h;
                if (tau_from_delta) {
                  const float v000 = dd(0, 0, 0), v100 = dd(1, 0, 0), v010 = dd(0, 1, 0), v110 = dd(1, 1, 0);
                  const float v001 = dd(0, 0, 1), v101 = dd(1, 0, 1), v011 = dd(0, 1, 1), v111 = dd(1, 1, 1);
                  GD[c][0] = ((v100 - v000) + (v110 - v010) + (v101 - v001) + (v111 - v011)) * inv4h;
                  GD[c][1] = ((v010 - v000) + (v110 - v100) + (v011 - v001) + (v111 - v101)) * inv4h;
                  GD[c][2] = ((v001 - v000) + (v101 - v100) + (v011 - v010) + (v111 - v110)) * inv4h;
                }
              }
            }
            const float exx = eps[0][0] + G[0][0], eyy = eps[1][1] + G[1][1], ezz = eps[2][2] + G[2][2];
            const float eyz = eps[1][2] + 0.5f * (G[1][2] + G[2][1]);
            const float exz = eps[0][2] + 0.5f * (G[0][2] + G[2][0]);
            const float exy = eps[0][1] + 0.5f * (G[0][1] + G[1][0]);
            const float tr = exx + eyy + ezz;
            const float sxx = lam * tr + 2.f * mu * exx, syy = lam * tr + 2.f * mu * eyy;
            const float szz = lam * tr + 2.f * mu * ezz;
            const float syz = 2.f * mu * eyz, sxz = 2.f * mu * exz, sxy = 2.f * mu * exy;
            Fs[0] += sxx * sx + sxy * sy + sxz * sz;
            Fs[1] += sxy * sx + syy * sy + syz * sz;
            Fs[2] += sxz * sx + syz * sy + szz * sz;
            if (tau_on) {
              const float (*GT)[3] = tau_from_delta ? GD : G;
              #pragma unroll
              for (int c = 0; c < 3; ++c)
                F0[c] += (2.f * mu0 + (c == 0 ? lam0 : 0.f)) * GT[c][0] * sx +
                         (2.f * mu0 + (c == 1 ? lam0 : 0.f)) * GT[c][1] * sy +
                         (2.f * mu0 + (c == 2 ? lam0 : 0.f)) * GT[c][2] * sz;
            }
            // each (voxel, integration point) counted once: TETRA2 T1 by corner 000, T2 by
            // corner 100; HEX1 by corner 000
            bool own;
            if constexpr (SCHEME == SCHEME_TETRA2) own = (dx == 0 && dy == 0 && dz == 0) || (dx == 1 && dy == 0 && dz == 0);
            else own = (dx == 0 && dy == 0 && dz == 0);
            if (own) {
              const float w = (SCHEME == SCHEME_TETRA2) ? 0.5f : 1.f;
              s2loc += w * (sxx * sxx + syy * syy + szz * szz + 2.f * (syz * syz + sxz * sxz + sxy * sxy));
            }
          }
        }
      }
      acc_s2 += (double)s2loc;
      // node boundary data
      const long long n = i + (long long)nnx * (j + (long long)nny * k);
      const uint8_t cm = a.cmask ? a.cmask[n] : 0;
      const int idx[3] = {i, j, k};
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        float invW = 1.f;
        bool dof = true;
        #pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (g.periodic[d]) continue;
          int f = -1;
          if (idx[d] == 0) f = 0;
          else if (idx[d] == g.nn[d] - 1) f = 1;
          if (f < 0) continue;
          const int t = g.bc[d][f][c];
          if (t == BC_D) dof = false;
          else if (t == BC_N) invW *= 2.f;
        }
        float pv = 0.f, a0v = 0.f;
        if (dof) {
          pv = -Fs[c] * c4h * invW;
          if (tau_on) a0v = F0[c] * c4h * invW;
        }
        const long long e = c * NN + n;
        const bool free_dof = dof && !((cm >> c) & 1);
        if (free_dof) acc_p2 += (double)(pv * pv);
        if (po) po[e] = pv;
        if (xo) xo[e] = pv + a0v;
        if (ro) {
          const float rv = dof ? (pv - gprev[e] + a0v) : 0.f;
          ro[e] = rv;
          if (free_dof) {
            #pragma unroll
            for (int q = 0; q < 4; ++q) acc_g[q] += (double)(rv * (q == rslot ? rv : Rk[q][e]));
          }
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // block reduction (FP64)
  double v[6] = {acc_s2, acc_p2, acc_g[0], acc_g[1], acc_g[2], acc_g[3]};
  const int warp = tid >> 5, lane = tid & 31;
  #pragma unroll
  for (int q = 0; q < 6; ++q) {
    double t = v[q];
    #pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) sRed[q][warp] = t;
  }
  __syncthreads();
  if (tid < 6) {
    double t = 0.0;
    for (int w = 0; w < FTX * FTY / 32; ++w) t += sRed[tid][w];
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    a.partials[6 * b + tid] = t;
  }
}

int residual_f32_zchunk(const GridDev& g) {
  long long bxy = (long long)((g.nn[0] + FTX - 1) / FTX) * ((g.nn[1] + FTY - 1) / FTY);
  long long want = 148LL * 4;
  long long zc = (g.nn[2] * bxy + want - 1) / want;
  if (zc < 2) zc = 2;
  if (zc > 32) zc = 32;
  return (int)zc;
}

int residual_f32_blocks(const GridDev& g) {
  int zc = residual_f32_zchunk(g);
  return ((g.nn[0] + FTX - 1) / FTX) * ((g.nn[1] + FTY - 1) / FTY) * ((g.nn[2] + zc - 1) / zc);
}

template <int SCHEME>
static int launch_f32_impl(const ResidualArgs& a, cudaStream_t s) {
  const int zc = residual_f32_zchunk(a.g);
  dim3 blk(FTX, FTY);
  dim3 grd((a.g.nn[0] + FTX - 1) / FTX, (a.g.nn[1] + FTY - 1) / FTY, (a.g.nn[2] + zc - 1) / zc);
  ResidualArgs aa = a;
  aa.zchunk = zc;
  const size_t sm = (size_t)3 * FNP * FPLANE * sizeof(float) + (size_t)FNP * FHY * FHX;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_residual_f32<SCHEME>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr = true;
  }
  k_residual_f32<SCHEME><<<grd, blk, sm, s>>>(aa);
  return (int)cudaGetLastError();
}

int launch_residual_f32(const ResidualArgs& a, cudaStream_t s) {
  if (a.g.scheme == SCHEME_TETRA2) return launch_f32_impl<SCHEME_TETRA2>(a, s);
  return launch_f32_impl<SCHEME_HEX1>(a, s);
}

}  // namespace dtt

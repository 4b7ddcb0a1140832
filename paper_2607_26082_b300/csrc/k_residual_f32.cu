// Stress / divergence / reference-operator kernel of the mixed path (same operator as
// k_residual.cu: Eq. 3 with the HEX1 / TETRA2 gradients of Section 3.1.1, the Paux
// reference medium of Section 3.2.3 and the symmetry weights W of Table 1), organised for
// FP32 throughput on B300:
//
//  * a CTA owns a 32 x 8 tile of node columns and marches along z one voxel layer at a
//    time; the layer between node planes L and L+1 is processed in two phases:
//      A. one thread per voxel of the 33 x 9 halo layer forms, once, the gradients of both
//         tetrahedra (TETRA2) or of the single point (HEX1), the stress sigma = C:(eps* +
//         sym grad u~) and the reference-medium flux tau_cd = (2 mu0 + lambda0 delta_cd)
//         d(.)_c/dx_d, and stores them in shared memory (structure of arrays);
//      B. one thread per node gathers, from the 4 voxels of the layer around its column,
//         the divergence contributions to node L (as their lower corner) and to node L+1
//         (as their upper corner); node L is then complete and its outputs are written;
//  * u~ (float-float hi / lo), the step Delta and the voxel phases of node planes L..L+2
//    sit in a 3-slot shared-memory ring filled with cp.async one plane ahead;
//  * in the Anderson difference form the kernel also forms the Gram row <R_{i-1}, R_k>
//    (k = 0..3) over the unconstrained DOFs; the projection kernels add the constrained
//    ones after they have shifted R_{i-1};
//  * no FP64 arithmetic inside the march: per-thread sums are compensated FP32 pairs
//    (TwoSum), converted to FP64 once per thread before the block reduction.
// Finite strain (FS = true, Section 5.2): phase A stores the 9 values of the first
// Piola-Kirchhoff stress Pi = F.S (St Venant-Kirchhoff, E = (H + H^T + H^T H) / 2 with
// H = eps* + grad u~, F = 1 + H, S = C : E) in place of sigma's 6, and phase B gathers
// its rows; the norm takes Pi : Pi.
// Partial sums per CTA (FP64): [sum w sigma:sigma, sum p^2, Gram 0..3].
#include "dtt_internal.cuh"

namespace dtt {

namespace {

constexpr int FTX = 32, FTY = 8;                 // node tile
constexpr int FVX = FTX + 1, FVY = FTY + 1;      // voxel layer with its low-side halo
constexpr int NVL = FVX * FVY;                   // 297 voxels per layer
constexpr int FTHREADS = 320;                    // >= NVL, multiple of 32
constexpr int FNP = 3;                           // node-plane ring slots
constexpr int FHX = FTX + 2, FHY = FTY + 2;      // node plane with halo (x0-1 .. x0+32)
constexpr int FPLANE = 3 * FHY * FHX;            // floats per plane (3 components)
template <bool FS> struct PointLayout {
  static constexpr int NS = FS ? 9 : 6;          // stress values per point (Pi or sigma)
  static constexpr int QV = NS + 9;              // plus tau 9
};

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
__device__ __forceinline__ int slot_of(int plane) { return ((plane % FNP) + FNP) % FNP; }

// compensated FP32 accumulator (TwoSum: s + c carries the sum to about FP32^2)
struct Acc2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ int sidx(int slot, int c, int ly, int lx) { return ((slot * 3 + c) * FHY + ly) * FHX + lx; }

// (ph + pl) - (qh + ql) from the pairs' differences, so that increments far below the
// FP32 resolution of u~ survive
__device__ __forceinline__ float fdiff(float ph, float pl, float qh, float ql) {
  return __fadd_rn(__fsub_rn(ph, qh), __fsub_rn(pl, ql));
}

// Reference flux tau = R0 : grad u, Paux or isotropic medium (Section 3.2.3).
__device__ __forceinline__ float ref_flux(const float (&Gm)[3][3], int c, int d, float lam0, float mu0, bool iso) {
  if (iso) return (c == d ? lam0 * (Gm[0][0] + Gm[1][1] + Gm[2][2]) : 0.f) + mu0 * (Gm[c][d] + Gm[d][c]);
  return (2.f * mu0 + (c == d ? lam0 : 0.f)) * Gm[c][d];
}

}  // namespace

template <int SCHEME, bool FS>
__global__ void __launch_bounds__(FTHREADS, 2)
k_residual_f32(ResidualArgs a) {
  constexpr int NPT = (SCHEME == SCHEME_TETRA2) ? 2 : 1;
  constexpr int NS = PointLayout<FS>::NS, QV = PointLayout<FS>::QV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sH = (float*)smem_raw;                 // [FNP][3][FHY][FHX] u~ hi
  float* sL = sH + FNP * FPLANE;                // u~ lo
  float* sD = sL + FNP * FPLANE;                // Delta
  float* sV = sD + FNP * FPLANE;                // [NPT * QV][NVL] point data of the current layer
  uint8_t* sP = (uint8_t*)(sV + NPT * QV * NVL);   // [FNP][FHY][FHX] voxel phases (layer of plane)
  __shared__ float sLam[MAX_PHASE], sMu[MAX_PHASE];
  __shared__ double sRed[6][FTHREADS / 32];

  if (a.ctrl && a.ctrl->done) return;
  const GridDev& g = a.g;
  const int tid = threadIdx.x;
  for (int q = tid; q < a.nphase; q += FTHREADS) {
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
  int tz_lo = -(1 << 29), tz_hi = 1 << 29;   // node planes where the flux's field can be non-zero
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
      #pragma unroll
      for (int q = 0; q < 4; ++q) Rk[q] = (const float*)a.rring[q];
      if (a.exact) {
        // R_{i-1} = p_i + A0 c_{i-1}: g_{i-1} is not needed, and A0 c vanishes unless the
        // CTA's nodes or their neighbours carry a correction; c lives on node planes
        // [zlo, zhi] of this tile, so only voxel layers zlo - 1 .. zhi carry its flux
        gprev = nullptr;
        const int2 zr = a.tile_z[blockIdx.y * gridDim.x + blockIdx.x];
        const int z1c = min((int)blockIdx.z * a.zchunk + a.zchunk, a.g.nn[2]);
        tau_on = zr.x <= zr.y && zr.y >= (int)blockIdx.z * a.zchunk - 1 && zr.x <= z1c;
        if (!tau_on) dfield = nullptr;
        tz_lo = zr.x;
        tz_hi = zr.y;
      }
    } else {
      tau_on = false;
    }
  } else {
    tau_on = false;
  }
  const float lam0 = a.f_lam0, mu0 = a.f_mu0;
  const bool iso = g.ref_iso != 0;
  const float inv2h = a.f_inv2h, inv4h = a.f_inv4h;
  const float c4h = inv4h;
  const float (&eps)[3][3] = a.f_eps;

  // ---- plane loader: node plane kk and the voxel phases of layer kk into ring slot.  Each
  // thread owns at most two positions of the 34 x 10 plane; their xy offsets are fixed for
  // the whole march.
  int nq = 0, q_off[2] = {0, 0};
  long long q_node[2] = {-1, -1}, q_vox[2] = {-1, -1};
  for (int q = tid; q < FHX * FHY; q += FTHREADS, ++nq) {
    const int lx = q % FHX, ly = q / FHX;
    q_off[nq] = ly * FHX + lx;
    const int gi = wrapi(x0 - 1 + lx, nnx, g.periodic[0]);
    const int gj = wrapi(y0 - 1 + ly, nny, g.periodic[1]);
    q_node[nq] = (gi >= 0 && gj >= 0) ? gi + (long long)nnx * gj : -1;
    const int vx = wrapi(x0 - 1 + lx, g.nvox[0], g.periodic[0]);
    const int vy = wrapi(y0 - 1 + ly, g.nvox[1], g.periodic[1]);
    q_vox[nq] = (vx >= 0 && vy >= 0) ? vx + (long long)g.nvox[0] * vy : -1;
  }
  const long long plane_n = (long long)nnx * nny, plane_v = (long long)g.nvox[0] * g.nvox[1];
  auto load_plane = [&](int kk) {
    const int slot = slot_of(kk);
    const int kw = wrapi(kk, nnz, g.periodic[2]);
    const int vz = wrapi(kk, g.nvox[2], g.periodic[2]);
    const bool dplane = dfield && kk >= tz_lo - 1 && kk <= tz_hi + 1;
    #pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m >= nq) break;
      const bool ok = kw >= 0 && q_node[m] >= 0;
      const long long n = ok ? q_node[m] + plane_n * kw : 0;
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int si = (slot * 3 + c) * FHY * FHX + q_off[m];
        if (ok) {
          cp_async4(&sH[si], a.uhi + c * NN + n);
          cp_async4(&sL[si], a.ulo + c * NN + n);
          if (dplane) cp_async4(&sD[si], dfield + c * NN + n);
          else sD[si] = 0.f;
        } else {
          sH[si] = 0.f;
          sL[si] = 0.f;
          sD[si] = 0.f;
        }
      }
      uint8_t ph = 255;   // 255 = no voxel
      if (vz >= 0 && q_vox[m] >= 0) ph = a.phase[q_vox[m] + plane_v * vz];
      sP[slot * FHY * FHX + q_off[m]] = ph;
    }
  };

  Acc2 acc_s2, acc_p2, acc_g[4];

  // node thread (i, j)
  const bool node_thread = tid < FTX * FTY;
  const int tx = tid % FTX, ty = tid / FTX;
  const int i = x0 + tx, j = y0 + ty;
  const bool active = node_thread && (i < nnx && j < nny);
  // voxel thread: local voxel (vlx, vly) = global voxel (x0 - 1 + vlx, y0 - 1 + vly); warps
  // 0..8 take the voxel rows' first 32 columns (one row per warp: bank-conflict free), the
  // first 9 lanes of warp 9 take column 32
  const bool vox_thread = tid < NVL;
  const int vlx = tid < FTX * FVY ? (tid % FTX) : FTX;
  const int vly = tid < FTX * FVY ? (tid / FTX) : (tid - FTX * FVY);
  const int vslot = vly * FVX + vlx;

  float Fc[3] = {0.f, 0.f, 0.f}, F0c[3] = {0.f, 0.f, 0.f};   // node plane L (complete after layer L)
  float Fn[3] = {0.f, 0.f, 0.f}, F0n[3] = {0.f, 0.f, 0.f};   // node plane L+1 (partial)

  load_plane(z0 - 1);
  load_plane(z0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();

  for (int L = z0 - 1; L < z1; ++L) {
    if (L + 2 <= z1) load_plane(L + 2);
    cp_async_commit();
    const int s0 = slot_of(L), s1 = slot_of(L + 1);
    // operands of node L's outputs, loaded now so that their latency overlaps phase A
    uint8_t cm = 0;
    float pg[3] = {0.f, 0.f, 0.f}, pr[4][3];
    const bool fin = active && L >= z0;
    const long long nL = (long long)i + (long long)nnx * (j + (long long)nny * L);
    if (fin) {
      cm = a.cmask ? a.cmask[nL] : 0;
      if (ro) {
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (gprev) pg[c] = gprev[c * NN + nL];
          #pragma unroll
          for (int q = 0; q < 4; ++q) pr[q][c] = (q == rslot) ? 0.f : Rk[q][c * NN + nL];
        }
      }
    }

    // the reference flux of this voxel layer (uniform over the CTA)
    const bool tau_L = tau_on && L >= tz_lo - 1 && L <= tz_hi;
    const bool need_gd = tau_L && tau_from_delta;
    // ---------------- phase A: point data of voxel layer L
    if (vox_thread) {
      const uint8_t ph = sP[(s0 * FHY + vly) * FHX + vlx];
      float* out = sV + vslot;
      if (ph == 255) {
        #pragma unroll
        for (int q = 0; q < NPT * QV; ++q) out[q * NVL] = 0.f;
      } else {
        const float lam = sLam[ph], mu = sMu[ph];
        // each voxel's sigma:sigma counted by the tile that holds its lower corner node
        const bool own = vlx >= 1 && vly >= 1 && L >= z0 && (x0 - 1 + vlx) < g.nvox[0] &&
                         (y0 - 1 + vly) < g.nvox[1] && L < g.nvox[2];
        const float w = (SCHEME == SCHEME_TETRA2) ? 0.5f : 1.f;
        // corner b = cx + 2 cy + 4 cz of the voxel, component c
        // corner b = cx + 2 cy + 4 cz, component c: the plane's base index plus a constant
        const int base0 = sidx(s0, 0, vly, vlx), base1 = sidx(s1, 0, vly, vlx);
        auto corner = [&](int b, int c) {
          return ((b >> 2) ? base1 : base0) + c * (FHY * FHX) + ((b >> 1) & 1) * FHX + (b & 1);
        };
        #pragma unroll
        for (int t = 0; t < NPT; ++t) {
          float G[3][3], GD[3][3];
          #pragma unroll
          for (int c = 0; c < 3; ++c) {
            if constexpr (SCHEME == SCHEME_TETRA2) {
              // T1 = {000, 110, 101, 011} = corners {0, 3, 5, 6}; T2 = {100, 010, 001, 111} =
              // corners {1, 2, 4, 7}; with (a, b, c, e) in that order the two gradients are
              //   T1: ((b-a) + (c-e), (b-a) - (c-e), (c-a) + (e-b)) / 2h
              //   T2: ((a-b) + (e-c), (e-c) - (a-b), (c-a) + (e-b)) / 2h
              const int ia = corner(t ? 1 : 0, c), ib = corner(t ? 2 : 3, c);
              const int ic = corner(t ? 4 : 5, c), ie = corner(t ? 7 : 6, c);
              const float ah = sH[ia], al = sL[ia], bh = sH[ib], bl = sL[ib];
              const float ch = sH[ic], cl = sL[ic], eh = sH[ie], el = sL[ie];
              const float d_ca = fdiff(ch, cl, ah, al), d_eb = fdiff(eh, el, bh, bl);
              G[c][2] = (d_ca + d_eb) * inv2h;
              if (t == 0) {
                const float d_ba = fdiff(bh, bl, ah, al), d_ce = fdiff(ch, cl, eh, el);
                G[c][0] = (d_ba + d_ce) * inv2h;
                G[c][1] = (d_ba - d_ce) * inv2h;
              } else {
                const float e_ab = fdiff(ah, al, bh, bl), e_ec = fdiff(eh, el, ch, cl);
                G[c][0] = (e_ab + e_ec) * inv2h;
                G[c][1] = (e_ec - e_ab) * inv2h;
              }
              if (need_gd) {
                const float A = sD[ia], B = sD[ib], Cc = sD[ic], E = sD[ie];
                GD[c][2] = ((Cc - A) + (E - B)) * inv2h;
                if (t == 0) {
                  GD[c][0] = ((B - A) + (Cc - E)) * inv2h;
                  GD[c][1] = ((B - A) - (Cc - E)) * inv2h;
                } else {
                  GD[c][0] = ((A - B) + (E - Cc)) * inv2h;
                  GD[c][1] = ((E - Cc) - (A - B)) * inv2h;
                }
              }
            } else {
              float uh[8], ul[8];
              #pragma unroll
              for (int b = 0; b < 8; ++b) {
                const int si = corner(b, c);
                uh[b] = sH[si];
                ul[b] = sL[si];
              }
              auto d = [&](int p, int q) { return fdiff(uh[p], ul[p], uh[q], ul[q]); };
              G[c][0] = (d(1, 0) + d(3, 2) + d(5, 4) + d(7, 6)) * inv4h;
              G[c][1] = (d(2, 0) + d(3, 1) + d(6, 4) + d(7, 5)) * inv4h;
              G[c][2] = (d(4, 0) + d(5, 1) + d(6, 2) + d(7, 3)) * inv4h;
              if (need_gd) {
                float ud[8];
                #pragma unroll
                for (int b = 0; b < 8; ++b) ud[b] = sD[corner(b, c)];
                GD[c][0] = ((ud[1] - ud[0]) + (ud[3] - ud[2]) + (ud[5] - ud[4]) + (ud[7] - ud[6])) * inv4h;
                GD[c][1] = ((ud[2] - ud[0]) + (ud[3] - ud[1]) + (ud[6] - ud[4]) + (ud[7] - ud[5])) * inv4h;
                GD[c][2] = ((ud[4] - ud[0]) + (ud[5] - ud[1]) + (ud[6] - ud[2]) + (ud[7] - ud[3])) * inv4h;
              }
            }
          }
          float* o = out + t * QV * NVL;
          if constexpr (FS) {
            float H[3][3], S[3][3];
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int dd = 0; dd < 3; ++dd) H[c][dd] = eps[c][dd] + G[c][dd];
            #pragma unroll
            for (int p = 0; p < 3; ++p)
              #pragma unroll
              for (int q = p; q < 3; ++q) {
                float v = H[p][q] + H[q][p];
                #pragma unroll
                for (int k = 0; k < 3; ++k) v = fmaf(H[k][p], H[k][q], v);
                S[p][q] = S[q][p] = 0.5f * v;   // E for now
              }
            const float tr = S[0][0] + S[1][1] + S[2][2];
            #pragma unroll
            for (int p = 0; p < 3; ++p)
              #pragma unroll
              for (int q = p; q < 3; ++q) S[p][q] = S[q][p] = 2.f * mu * S[p][q] + (p == q ? lam * tr : 0.f);
            float s2 = 0.f;
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int dd = 0; dd < 3; ++dd) {
                float v = S[c][dd];
                #pragma unroll
                for (int k = 0; k < 3; ++k) v = fmaf(H[c][k], S[k][dd], v);
                o[(3 * c + dd) * NVL] = v;
                s2 = fmaf(v, v, s2);
              }
            if (tau_L) {
              #pragma unroll
              for (int c = 0; c < 3; ++c)
                #pragma unroll
                for (int dd = 0; dd < 3; ++dd)
                  o[(NS + 3 * c + dd) * NVL] =
                      (tau_from_delta ? ref_flux(GD, c, dd, lam0, mu0, iso) : ref_flux(G, c, dd, lam0, mu0, iso));
            }
            if (own) acc_s2.add(w * s2);
            continue;
          }
          const float exx = eps[0][0] + G[0][0], eyy = eps[1][1] + G[1][1];
          const float ezz = eps[2][2] + G[2][2];
          const float eyz = eps[1][2] + 0.5f * (G[1][2] + G[2][1]);
          const float exz = eps[0][2] + 0.5f * (G[0][2] + G[2][0]);
          const float exy = eps[0][1] + 0.5f * (G[0][1] + G[1][0]);
          const float tr = exx + eyy + ezz;
          const float sxx = lam * tr + 2.f * mu * exx, syy = lam * tr + 2.f * mu * eyy;
          const float szz = lam * tr + 2.f * mu * ezz;
          const float syz = 2.f * mu * eyz, sxz = 2.f * mu * exz, sxy = 2.f * mu * exy;
          o[0 * NVL] = sxx;
          o[1 * NVL] = syy;
          o[2 * NVL] = szz;
          o[3 * NVL] = syz;
          o[4 * NVL] = sxz;
          o[5 * NVL] = sxy;
          if (tau_L) {
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int dd = 0; dd < 3; ++dd)
                o[(NS + 3 * c + dd) * NVL] =
                    (tau_from_delta ? ref_flux(GD, c, dd, lam0, mu0, iso) : ref_flux(G, c, dd, lam0, mu0, iso));
          }
          if (own) acc_s2.add(w * (sxx * sxx + syy * syy + szz * szz + 2.f * (syz * syz + sxz * sxz + sxy * sxy)));
        }
      }
    }
    __syncthreads();

    // ---------------- phase B: gather into node L (lower corner) and node L+1 (upper corner)
    if (active) {
      #pragma unroll
      for (int ey = 0; ey < 2; ++ey) {
        #pragma unroll
        for (int ex = 0; ex < 2; ++ex) {
          const int v = (ty + ey) * FVX + (tx + ex);
          const int dx = 1 - ex, dy = 1 - ey;
          const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f;
          // node L is corner (dx, dy, 0) of the voxel, node L+1 its corner (dx, dy, 1);
          // TETRA2: the point whose tetrahedron holds the corner (T1 = even parity)
          const int tlo = (SCHEME == SCHEME_TETRA2) ? ((dx + dy) & 1) : 0;
          const int thi = (SCHEME == SCHEME_TETRA2) ? (1 - tlo) : 0;
          auto gather = [&](float (&F)[3], float (&F0)[3], int t, float sz) {
            const float* q = sV + t * QV * NVL + v;
            if constexpr (FS) {
              #pragma unroll
              for (int c = 0; c < 3; ++c)
                F[c] += q[(3 * c) * NVL] * sx + q[(3 * c + 1) * NVL] * sy + q[(3 * c + 2) * NVL] * sz;
            } else {
              const float sxx = q[0], syy = q[NVL], szz = q[2 * NVL];
              const float syz = q[3 * NVL], sxz = q[4 * NVL], sxy = q[5 * NVL];
              F[0] += sxx * sx + sxy * sy + sxz * sz;
              F[1] += sxy * sx + syy * sy + syz * sz;
              F[2] += sxz * sx + syz * sy + szz * sz;
            }
            if (tau_L) {
              #pragma unroll
              for (int c = 0; c < 3; ++c)
                F0[c] += q[(NS + 3 * c) * NVL] * sx + q[(NS + 1 + 3 * c) * NVL] * sy + q[(NS + 2 + 3 * c) * NVL] * sz;
            }
          };
          gather(Fc, F0c, tlo, -1.f);
          gather(Fn, F0n, thi, 1.f);
        }
      }
      // node plane L is complete
      if (fin) {
        const int k = L;
        const long long n = nL;
        const int idx[3] = {i, j, k};
        // nodes on no non-periodic face (most of them) skip the per-component face checks
        bool face = false;
        #pragma unroll
        for (int d = 0; d < 3; ++d) face |= !g.periodic[d] && (idx[d] == 0 || idx[d] == g.nn[d] - 1);
        float p2loc = 0.f, gloc[4] = {0.f, 0.f, 0.f, 0.f};
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          float invW = 1.f;
          bool dof = true;
          if (face) {
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
          }
          float pv = 0.f, a0v = 0.f;
          if (dof) {
            pv = -Fc[c] * c4h * invW;
            if (tau_on) a0v = F0c[c] * c4h * invW;
          }
          const long long e = c * NN + n;
          const bool free_dof = dof && !((cm >> c) & 1);
          if (free_dof) p2loc = fmaf(pv, pv, p2loc);
          if (po) po[e] = pv;
          if (xo) xo[e] = pv + a0v;
          if (ro) {
            const float rv = dof ? (pv - pg[c] + a0v) : 0.f;
            ro[e] = rv;
            if (free_dof) {
              #pragma unroll
              for (int q = 0; q < 4; ++q) gloc[q] = fmaf(rv, (q == rslot ? rv : pr[q][c]), gloc[q]);
            }
          }
        }
        acc_p2.add(p2loc);
        if (ro) {
          #pragma unroll
          for (int q = 0; q < 4; ++q) acc_g[q].add(gloc[q]);
        }
      }
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        Fc[c] = Fn[c];
        F0c[c] = F0n[c];
        Fn[c] = 0.f;
        F0n[c] = 0.f;
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // block reduction: compensated FP32 pairs across the warp, FP64 across warps
  Acc2 v[6] = {acc_s2, acc_p2, acc_g[0], acc_g[1], acc_g[2], acc_g[3]};
  const int warp = tid >> 5, lane = tid & 31;
  #pragma unroll
  for (int q = 0; q < 6; ++q) {
    Acc2 t = v[q];
    #pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float os = __shfl_down_sync(0xffffffffu, t.s, off);
      const float oc = __shfl_down_sync(0xffffffffu, t.c, off);
      t.add(os);
      t.c += oc;
    }
    if (lane == 0) sRed[q][warp] = t.value();
  }
  __syncthreads();
  if (tid < 6) {
    double t = 0.0;
    for (int w = 0; w < FTHREADS / 32; ++w) t += sRed[tid][w];
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    a.partials[6 * b + tid] = t;
  }
}

namespace {
int resident_ctas() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = 2 * sms;
  }
  return cached;
}
}  // namespace

// z planes per CTA: about two waves of resident CTAs, at least 4 planes per CTA (each CTA
// also processes the voxel layer below its first plane).
int residual_f32_zchunk(const GridDev& g) {
  if (g.zc_override > 0) return g.zc_override;
  long long bxy = (long long)((g.nn[0] + FTX - 1) / FTX) * ((g.nn[1] + FTY - 1) / FTY);
  long long want = 2LL * resident_ctas();
  long long zc = (g.nn[2] * bxy + want - 1) / want;
  if (zc < 4) zc = 4;
  if (zc > 64) zc = 64;
  return (int)zc;
}

int residual_f32_tile(int axis) { return axis == 0 ? FTX : FTY; }

int residual_f32_blocks(const GridDev& g) {
  int zc = residual_f32_zchunk(g);
  return ((g.nn[0] + FTX - 1) / FTX) * ((g.nn[1] + FTY - 1) / FTY) * ((g.nn[2] + zc - 1) / zc);
}

template <int SCHEME, bool FS>
static int launch_f32_impl(const ResidualArgs& a, cudaStream_t s) {
  const int zc = residual_f32_zchunk(a.g);
  dim3 grd((a.g.nn[0] + FTX - 1) / FTX, (a.g.nn[1] + FTY - 1) / FTY, (a.g.nn[2] + zc - 1) / zc);
  ResidualArgs aa = a;
  aa.zchunk = zc;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) aa.f_eps[p][q] = (float)a.eps[p][q];
  aa.f_lam0 = (float)a.lam0;
  aa.f_mu0 = (float)a.mu0;
  aa.f_inv2h = (float)(1.0 / (2.0 * a.g.h));
  aa.f_inv4h = (float)(1.0 / (4.0 * a.g.h));
  constexpr int NPT = (SCHEME == SCHEME_TETRA2) ? 2 : 1;
  constexpr int QV = PointLayout<FS>::QV;
  const size_t sm = (size_t)3 * FNP * FPLANE * sizeof(float) + (size_t)NPT * QV * NVL * sizeof(float) +
                    (size_t)FNP * FHY * FHX;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_residual_f32<SCHEME, FS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr = true;
  }
  k_residual_f32<SCHEME, FS><<<grd, FTHREADS, sm, s>>>(aa);
  return (int)cudaGetLastError();
}

int launch_residual_f32(const ResidualArgs& a, cudaStream_t s) {
  const bool fs = a.g.finite_strain != 0;
  if (a.g.scheme == SCHEME_TETRA2)
    return fs ? launch_f32_impl<SCHEME_TETRA2, true>(a, s) : launch_f32_impl<SCHEME_TETRA2, false>(a, s);
  return fs ? launch_f32_impl<SCHEME_HEX1, true>(a, s) : launch_f32_impl<SCHEME_HEX1, false>(a, s);
}

}  // namespace dtt

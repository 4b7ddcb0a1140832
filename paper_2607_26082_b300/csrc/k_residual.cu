// Fused stress / divergence / reference-operator kernel (Eq. 3, Algorithm 1: sigma,
// p = div_D sigma, p~ = p - div_D(R0 : grad_D u~)).
//
// Discretisation (Section 3.1.1, Fig. 1): nodes at integer positions; per voxel either one
// integration point (HEX1: grad_d u = (1/4h) sum_8 s_d u, weight 1) or two (TETRA2: one
// per inscribed tetrahedron, T1 = even-parity corners, T2 = odd-parity corners,
// grad_d u = (1/2h) sum_4 s_d u, weight 1/2), s_d = +1 on the voxel's upper side in d.
// div_D is the negative adjoint of grad_D; at a node it reads
//     p_c = -(1/(4h W_c)) * sum over the adjacent voxels of sum_d sigma_cd s_d(corner)
// (w * coefficient = 1/(4h) for both schemes), W_c = 2^-k for a node on k Neumann faces
// of component c (the symmetry-extension weight of Table 1; face reactions halved and
// edge reactions quartered as in Section 4.1.3), p_c = 0 on Dirichlet faces of c.
// The Paux reference medium (Section 3.2.3) R0 : grad u = lambda0 (grad u (.) I)
// + 2 mu0 grad u enters through tau0_cd = (2 mu0 + lambda0 delta_cd) grad_d u_c.
//
// Finite strain (FS = true; Section 5.2, Eq. 29): the divergence acts on the first
// Piola-Kirchhoff stress Pi = F.S of a St Venant-Kirchhoff material, S = C : E with
// E = (F^T F - 1) / 2 formed as (H + H^T + H^T H) / 2, H = eps* + grad u~, F = 1 + H (the
// same quantity without the cancellation of F^T F - 1 at small strain).  Pi is not
// symmetric: 9 values per point, gathered row by row; the Eq. 5 norm takes Pi : Pi.
//
// Modes: 0 (operator) writes p and p~ = p + A0 u~; 2 writes p only; 1 (Anderson on p~ in
// difference form) writes p into the p ring and, from the second iteration on, the
// Anderson residual R_{i-1} = p_i - g_{i-1} + A0 Delta_{i-1} (Delta = last step of u~,
// g = last Green input), which equals p~_i - S_{i-1} without forming either large term.
//
// B300 layout: one CTA owns a 32 x 4 tile of nodes in (x, y) and marches along z
// through a chunk of planes.  It keeps two node planes of u~ and two voxel planes of
// integration-point tensors (sigma: 6 values, tau0: 9 values per point) in shared memory,
// so each voxel's stress is evaluated once per CTA (plus a one-voxel halo) and every
// global access is a coalesced row of the tile.  The kernel writes p and p~ (nodal,
// component-major) and FP64 per-block partial sums of sum w sigma:sigma (each voxel
// counted by the CTA owning its lower corner) and sum p^2 over unconstrained DOFs.
#include "dtt_internal.cuh"

namespace dtt {

constexpr int RTX = 32;   // tile width (x nodes)
constexpr int RTY = 4;    // tile height (y nodes)
constexpr int RZC_MAX = 16;   // z planes per CTA (at most)
constexpr int NX2 = RTX + 2, NY2 = RTY + 2;   // node halo tile
constexpr int VX = RTX + 1, VY = RTY + 1;     // voxel tile

template <bool MIX> struct NodeV;
template <> struct NodeV<false> { double v; };
template <> struct NodeV<true> { float hi, lo; };

__device__ __forceinline__ double ndiff(const NodeV<false>& a, const NodeV<false>& b) { return a.v - b.v; }
__device__ __forceinline__ float ndiff(const NodeV<true>& a, const NodeV<true>& b) {
  return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

template <typename T, int NIP, int NS> struct VoxV {
  T sig[NIP][NS];   // NS = 6: sigma xx yy zz yz xz xy; NS = 9: Pi row c, column d
  T tau[NIP][9];    // row c, column d
};

__device__ __forceinline__ int wrap_or_neg(int i, int n, int per) {
  if (per) { i %= n; if (i < 0) i += n; return i; }
  return (i < 0 || i >= n) ? -1 : i;
}

// Node-side boundary data: DOF flag and 1/W for component c at node (i,j,k).
__device__ __forceinline__ double node_invW(const GridDev& g, int c, int i, int j, int k, bool& dof) {
  double invW = 1.0;
  dof = true;
  const int idx[3] = {i, j, k};
  #pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (g.periodic[d]) continue;
    int f = -1;
    if (idx[d] == 0) f = 0;
    else if (idx[d] == g.nn[d] - 1) f = 1;
    if (f < 0) continue;
    int t = g.bc[d][f][c];
    if (t == BC_D) dof = false;
    else if (t == BC_N) invW *= 2.0;
  }
  return invW;
}

// Reference flux tau = R0 : grad u (row c, column d) of the Paux medium,
// (2 mu0 + lambda0 delta_cd) grad_d u_c, or of the isotropic medium,
// lambda0 delta_cd tr(grad u) + mu0 (grad_d u_c + grad_c u_d) (Section 3.2.3).
template <typename T>
__device__ __forceinline__ T ref_flux(const T (&Gm)[3][3], int c, int d, T lam0, T mu0, bool iso) {
  if (iso) return (c == d ? lam0 * (Gm[0][0] + Gm[1][1] + Gm[2][2]) : (T)0) + mu0 * (Gm[c][d] + Gm[d][c]);
  return ((T)2 * mu0 + (c == d ? lam0 : (T)0)) * Gm[c][d];
}

template <typename T, bool MIX, int SCHEME, bool FS>
__global__ void __launch_bounds__(RTX * RTY)
k_residual(ResidualArgs a) {
  constexpr int NIP = (SCHEME == SCHEME_TETRA2) ? 2 : 1;
  constexpr int NS = FS ? 9 : 6;
  using Vox = VoxV<T, NIP, NS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sLam = (double*)smem_raw;
  double* sMu = sLam + MAX_PHASE;
  double (*sRed)[RTX * RTY / 32] = (double (*)[RTX * RTY / 32])(sMu + MAX_PHASE);
  Vox (*sV)[VY][VX] = (Vox (*)[VY][VX])(smem_raw + 2 * MAX_PHASE * 8 + 2 * (RTX * RTY / 32) * 8);
  NodeV<MIX> (*sU)[3][NY2][NX2] = (NodeV<MIX> (*)[3][NY2][NX2])((unsigned char*)sV + 2 * VY * VX * sizeof(Vox));
  T (*sD)[3][NY2][NX2] = (T (*)[3][NY2][NX2])((unsigned char*)sU + 2 * 3 * NY2 * NX2 * sizeof(NodeV<MIX>));

  const GridDev& g = a.g;
  if (a.ctrl && a.ctrl->done) return;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
  for (int q = tid; q < a.nphase; q += RTX * RTY) { sLam[q] = a.lam[q]; sMu[q] = a.mu[q]; }

  const int x0 = blockIdx.x * RTX, y0 = blockIdx.y * RTY;
  const int zc = a.zchunk;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, g.nn[2]);
  const long long NN = g.nnodes;
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];
  T* xo = nullptr;
  T* po = (T*)a.pout;
  T* ro = nullptr;
  const T* gprev = nullptr;
  const T* dfield = nullptr;
  bool tau_on = true;          // compute the reference-operator term
  if (a.mode == 0) {
    xo = (T*)a.xout;
  } else if (a.mode == 1) {
    const int il = a.ctrl->i_local;
    po = (T*)a.pring[il % 4];
    if (il > 0) {
      ro = (T*)a.rring[(il - 1) % 4];
      gprev = (const T*)a.gring[(il - 1) % 4];
      dfield = (const T*)a.dfield;
    } else {
      tau_on = false;
    }
  } else {
    tau_on = false;
  }
  const double h = g.h;
  const T lam0 = (T)a.lam0, mu0 = (T)a.mu0;
  const bool iso = g.ref_iso != 0;
  T eps[3][3];
  #pragma unroll
  for (int p = 0; p < 3; ++p)
    #pragma unroll
    for (int q = 0; q < 3; ++q) eps[p][q] = (T)a.eps[p][q];

  double acc_s2 = 0.0, acc_p2 = 0.0;

  // load one node plane kk into ring slot sl
  auto load_nodes = [&](int kk, int sl) {
    int kw = wrap_or_neg(kk, nnz, g.periodic[2]);
    for (int q = tid; q < NX2 * NY2; q += RTX * RTY) {
      int lx = q % NX2, ly = q / NX2;
      int gi = wrap_or_neg(x0 - 1 + lx, nnx, g.periodic[0]);
      int gj = wrap_or_neg(y0 - 1 + ly, nny, g.periodic[1]);
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        NodeV<MIX> v;
        if (kw >= 0 && gi >= 0 && gj >= 0) {
          long long n = (long long)c * NN + gi + (long long)nnx * (gj + (long long)nny * kw);
          if constexpr (MIX) { v.hi = a.uhi[n]; v.lo = a.ulo[n]; }
          else { v.v = a.u64[n]; }
        } else {
          if constexpr (MIX) { v.hi = 0.f; v.lo = 0.f; } else { v.v = 0.0; }
        }
        sU[sl][c][ly][lx] = v;
        if (dfield) {
          T dv = (T)0;
          if (kw >= 0 && gi >= 0 && gj >= 0)
            dv = dfield[(long long)c * NN + gi + (long long)nnx * (gj + (long long)nny * kw)];
          sD[sl][c][ly][lx] = dv;
        }
      }
    }
  };

  // evaluate voxel plane vz from node slots (lower sl0, upper sl1) into voxel slot vs
  auto eval_voxels = [&](int vz, int sl0, int sl1, int vs, bool count_norm) {
    int vzw = wrap_or_neg(vz, g.nvox[2], g.periodic[2]);
    for (int q = tid; q < VX * VY; q += RTX * RTY) {
      int lx = q % VX, ly = q / VX;       // voxel local (lx, ly) has lower corner node (lx, ly) in sU
      int vx = x0 - 1 + lx, vy = y0 - 1 + ly;
      int vxw = wrap_or_neg(vx, g.nvox[0], g.periodic[0]);
      int vyw = wrap_or_neg(vy, g.nvox[1], g.periodic[1]);
      Vox& V = sV[vs][ly][lx];
      if (vxw < 0 || vyw < 0 || vzw < 0 || !tau_on) {
        #pragma unroll
        for (int t = 0; t < NIP; ++t)
          #pragma unroll
          for (int e = 0; e < 9; ++e) V.tau[t][e] = (T)0;
      }
      if (vxw < 0 || vyw < 0 || vzw < 0) {
        #pragma unroll
        for (int t = 0; t < NIP; ++t) {
          #pragma unroll
          for (int e = 0; e < NS; ++e) V.sig[t][e] = (T)0;
          #pragma unroll
          for (int e = 0; e < 9; ++e) V.tau[t][e] = (T)0;
        }
        continue;
      }
      int ph = a.phase[vxw + (long long)g.nvox[0] * (vyw + (long long)g.nvox[1] * vzw)];
      const T lam = (T)sLam[ph], mu = (T)sMu[ph];
      const T inv2h = (T)(1.0 / (2.0 * h));
      T G[NIP][3][3];
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        // corners u(dx,dy,dz)
        const NodeV<MIX>& u000 = sU[sl0][c][ly][lx];
        const NodeV<MIX>& u100 = sU[sl0][c][ly][lx + 1];
        const NodeV<MIX>& u010 = sU[sl0][c][ly + 1][lx];
        const NodeV<MIX>& u110 = sU[sl0][c][ly + 1][lx + 1];
        const NodeV<MIX>& u001 = sU[sl1][c][ly][lx];
        const NodeV<MIX>& u101 = sU[sl1][c][ly][lx + 1];
        const NodeV<MIX>& u011 = sU[sl1][c][ly + 1][lx];
        const NodeV<MIX>& u111 = sU[sl1][c][ly + 1][lx + 1];
        if constexpr (SCHEME == SCHEME_TETRA2) {
          // T1 = {000, 110, 101, 011}
          T d_ba = (T)ndiff(u110, u000), d_ce = (T)ndiff(u101, u011);
          T d_ca = (T)ndiff(u101, u000), d_eb = (T)ndiff(u011, u110);
          G[0][c][0] = (d_ba + d_ce) * inv2h;
          G[0][c][1] = (d_ba - d_ce) * inv2h;
          G[0][c][2] = (d_ca + d_eb) * inv2h;
          // T2 = {100, 010, 001, 111}
          T e_ab = (T)ndiff(u100, u010), e_ec = (T)ndiff(u111, u001);
          T e_ca = (T)ndiff(u001, u100), e_eb = (T)ndiff(u111, u010);
          G[NIP - 1][c][0] = (e_ab + e_ec) * inv2h;
          G[NIP - 1][c][1] = (e_ec - e_ab) * inv2h;
          G[NIP - 1][c][2] = (e_ca + e_eb) * inv2h;
        } else {
          const T inv4h = (T)(1.0 / (4.0 * h));
          T dx = (T)ndiff(u100, u000) + (T)ndiff(u110, u010) + (T)ndiff(u101, u001) + (T)ndiff(u111, u011);
          T dy = (T)ndiff(u010, u000) + (T)ndiff(u110, u100) + (T)ndiff(u011, u001) + (T)ndiff(u111, u101);
          T dzz = (T)ndiff(u001, u000) + (T)ndiff(u101, u100) + (T)ndiff(u011, u010) + (T)ndiff(u111, u110);
          G[0][c][0] = dx * inv4h;
          G[0][c][1] = dy * inv4h;
          G[0][c][2] = dzz * inv4h;
        }
      }
      // each voxel counted once: by the CTA owning its lower-corner node, and only for its
      // unwrapped index (a periodic axis shorter than the tile wraps halo voxels)
      bool own = count_norm && lx >= 1 && ly >= 1 && (vx < x0 + RTX) && (vy < y0 + RTY) &&
                 vx < g.nvox[0] && vy < g.nvox[1];
      #pragma unroll
      for (int t = 0; t < NIP; ++t) {
        if constexpr (FS) {
          T H[3][3], E[3][3], S[3][3];
          #pragma unroll
          for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d) H[c][d] = eps[c][d] + G[t][c][d];
          #pragma unroll
          for (int p = 0; p < 3; ++p)
            #pragma unroll
            for (int q = p; q < 3; ++q) {
              T v = H[p][q] + H[q][p];
              #pragma unroll
              for (int k = 0; k < 3; ++k) v += H[k][p] * H[k][q];
              E[p][q] = E[q][p] = (T)0.5 * v;
            }
          const T tr = E[0][0] + E[1][1] + E[2][2];
          #pragma unroll
          for (int p = 0; p < 3; ++p)
            #pragma unroll
            for (int q = 0; q < 3; ++q) S[p][q] = (T)2 * mu * E[p][q] + (p == q ? lam * tr : (T)0);
          double s2 = 0.0;
          #pragma unroll
          for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
              T v = S[c][d];
              #pragma unroll
              for (int k = 0; k < 3; ++k) v += H[c][k] * S[k][d];
              V.sig[t][3 * c + d] = v;
              s2 += (double)v * v;
            }
          if (tau_on && !dfield) {
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int d = 0; d < 3; ++d)
                V.tau[t][3 * c + d] = ref_flux<T>(G[t], c, d, lam0, mu0, iso);
          }
          if (own) acc_s2 += ((NIP == 2) ? 0.5 : 1.0) * s2;
          continue;
        }
        T exx = eps[0][0] + G[t][0][0], eyy = eps[1][1] + G[t][1][1], ezz = eps[2][2] + G[t][2][2];
        T eyz = eps[1][2] + (T)0.5 * (G[t][1][2] + G[t][2][1]);
        T exz = eps[0][2] + (T)0.5 * (G[t][0][2] + G[t][2][0]);
        T exy = eps[0][1] + (T)0.5 * (G[t][0][1] + G[t][1][0]);
        T tr = exx + eyy + ezz;
        T sxx = lam * tr + (T)2 * mu * exx, syy = lam * tr + (T)2 * mu * eyy, szz = lam * tr + (T)2 * mu * ezz;
        T syz = (T)2 * mu * eyz, sxz = (T)2 * mu * exz, sxy = (T)2 * mu * exy;
        V.sig[t][0] = sxx; V.sig[t][1] = syy; V.sig[t][2] = szz;
        V.sig[t][3] = syz; V.sig[t][4] = sxz; V.sig[t][5] = sxy;
        if (tau_on && !dfield) {
          #pragma unroll
          for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d)
              V.tau[t][3 * c + d] = ref_flux<T>(G[t], c, d, lam0, mu0, iso);
        }
        if (own) {
          double w = (NIP == 2) ? 0.5 : 1.0;
          double s2 = (double)sxx * sxx + (double)syy * syy + (double)szz * szz +
                      2.0 * ((double)syz * syz + (double)sxz * sxz + (double)sxy * sxy);
          acc_s2 += w * s2;
        }
      }
      if (dfield) {
        // reference-operator tensor of the step Delta (plain differences: Delta is small)
        T GD[NIP][3][3];
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T u000 = sD[sl0][c][ly][lx], u100 = sD[sl0][c][ly][lx + 1];
          const T u010 = sD[sl0][c][ly + 1][lx], u110 = sD[sl0][c][ly + 1][lx + 1];
          const T u001 = sD[sl1][c][ly][lx], u101 = sD[sl1][c][ly][lx + 1];
          const T u011 = sD[sl1][c][ly + 1][lx], u111 = sD[sl1][c][ly + 1][lx + 1];
          if constexpr (SCHEME == SCHEME_TETRA2) {
            T d_ba = u110 - u000, d_ce = u101 - u011, d_ca = u101 - u000, d_eb = u011 - u110;
            GD[0][c][0] = (d_ba + d_ce) * inv2h;
            GD[0][c][1] = (d_ba - d_ce) * inv2h;
            GD[0][c][2] = (d_ca + d_eb) * inv2h;
            T e_ab = u100 - u010, e_ec = u111 - u001, e_ca = u001 - u100, e_eb = u111 - u010;
            GD[NIP - 1][c][0] = (e_ab + e_ec) * inv2h;
            GD[NIP - 1][c][1] = (e_ec - e_ab) * inv2h;
            GD[NIP - 1][c][2] = (e_ca + e_eb) * inv2h;
          } else {
            const T inv4h = (T)(1.0 / (4.0 * h));
            GD[0][c][0] = ((u100 - u000) + (u110 - u010) + (u101 - u001) + (u111 - u011)) * inv4h;
            GD[0][c][1] = ((u010 - u000) + (u110 - u100) + (u011 - u001) + (u111 - u101)) * inv4h;
            GD[0][c][2] = ((u001 - u000) + (u101 - u100) + (u011 - u010) + (u111 - u110)) * inv4h;
          }
        }
        #pragma unroll
        for (int t = 0; t < NIP; ++t)
          #pragma unroll
          for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int d = 0; d < 3; ++d)
              V.tau[t][3 * c + d] = ref_flux<T>(GD[t], c, d, lam0, mu0, iso);
      }
    }
  };

  // prologue: node planes z0-1, z0 ; voxel plane z0-1
  int cur = 0;   // node slot holding plane k (current), other slot gets k+1
  load_nodes(z0 - 1, 1);
  load_nodes(z0, 0);
  __syncthreads();
  int vprev = 1;  // voxel slot holding plane k-1
  eval_voxels(z0 - 1, 1, 0, vprev, false);
  __syncthreads();

  for (int k = z0; k < z1; ++k) {
    int nxt = cur ^ 1;
    load_nodes(k + 1, nxt);
    __syncthreads();
    int vcur = vprev ^ 1;
    eval_voxels(k, cur, nxt, vcur, true);
    __syncthreads();
    // gather for node (x0+tx, y0+ty, k)
    int i = x0 + tx, j = y0 + ty;
    if (i < nnx && j < nny) {
      T Fs[3] = {(T)0, (T)0, (T)0}, F0[3] = {(T)0, (T)0, (T)0};
      #pragma unroll
      for (int ez = 0; ez < 2; ++ez) {
        const int vs = ez ? vcur : vprev;
        #pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
          #pragma unroll
          for (int ex = 0; ex < 2; ++ex) {
            // voxel with lower corner (i-1+ex, j-1+ey, k-1+ez): local (tx+ex, ty+ey)
            const Vox& V = sV[vs][ty + ey][tx + ex];
            // node is corner delta = (1-ex, 1-ey, 1-ez) of that voxel
            const int dx = 1 - ex, dy = 1 - ey, dzc = 1 - ez;
            const T sx = dx ? (T)1 : (T)-1, sy = dy ? (T)1 : (T)-1, sz = dzc ? (T)1 : (T)-1;
            const int t = (NIP == 2) ? ((dx + dy + dzc) & 1) : 0;
            if constexpr (FS) {
              #pragma unroll
              for (int c = 0; c < 3; ++c)
                Fs[c] += V.sig[t][3 * c] * sx + V.sig[t][3 * c + 1] * sy + V.sig[t][3 * c + 2] * sz;
            } else {
              // sigma rows: x: (xx, xy, xz), y: (xy, yy, yz), z: (xz, yz, zz)
              Fs[0] += V.sig[t][0] * sx + V.sig[t][5] * sy + V.sig[t][4] * sz;
              Fs[1] += V.sig[t][5] * sx + V.sig[t][1] * sy + V.sig[t][3] * sz;
              Fs[2] += V.sig[t][4] * sx + V.sig[t][3] * sy + V.sig[t][2] * sz;
            }
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              F0[c] += V.tau[t][3 * c] * sx + V.tau[t][3 * c + 1] * sy + V.tau[t][3 * c + 2] * sz;
          }
        }
      }
      const long long n = i + (long long)nnx * (j + (long long)nny * k);
      uint8_t cm = a.cmask ? a.cmask[n] : 0;
      const T c4h = (T)(1.0 / (4.0 * h));
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        bool dof;
        double invW = node_invW(g, c, i, j, k, dof);
        T pv = (T)0, a0v = (T)0;
        if (dof) {
          pv = -Fs[c] * c4h * (T)invW;
          if (tau_on) a0v = F0[c] * c4h * (T)invW;
          if (!((cm >> c) & 1)) acc_p2 += (double)pv * (double)pv;
        }
        const long long e = (long long)c * NN + n;
        if (po) po[e] = pv;
        if (xo) xo[e] = pv + a0v;
        if (ro) ro[e] = dof ? (pv - gprev[e] + a0v) : (T)0;
      }
    }
    cur = nxt;
    vprev = vcur;
    // the next iteration overwrites slot `nxt^1` (= old cur) and voxel slot vprev^1: both
    // were last read before the __syncthreads at the top of the next iteration's eval.
    __syncthreads();
  }

  // block reduction of the two partial sums (FP64)
  #pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc_s2 += __shfl_down_sync(0xffffffffu, acc_s2, off);
    acc_p2 += __shfl_down_sync(0xffffffffu, acc_p2, off);
  }
  const int warp = tid >> 5, lane = tid & 31;
  if (lane == 0) { sRed[0][warp] = acc_s2; sRed[1][warp] = acc_p2; }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0, p = 0.0;
    for (int w = 0; w < RTX * RTY / 32; ++w) { s += sRed[0][w]; p += sRed[1][w]; }
    long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    double* o = a.partials + RES_STRIDE * b;
    o[0] = s;
    o[1] = p;
    for (int q = 2; q < RES_STRIDE; ++q) o[q] = 0.0;
  }
}

// z planes per CTA: long chunks amortise the one-plane halo, short ones give small grids
// enough CTAs to fill the 148 SMs (target ~4 CTAs per SM).
int residual_zchunk(const GridDev& g) {
  if (g.zc_override > 0) return g.zc_override < RZC_MAX ? g.zc_override : RZC_MAX;
  long long bxy = (long long)((g.nn[0] + RTX - 1) / RTX) * ((g.nn[1] + RTY - 1) / RTY);
  long long want = 148LL * 4;
  long long zc = (g.nn[2] * bxy + want - 1) / want;
  if (zc < 2) zc = 2;
  if (zc > RZC_MAX) zc = RZC_MAX;
  return (int)zc;
}

int residual_blocks(const GridDev& g) {
  int zc = residual_zchunk(g);
  int bx = (g.nn[0] + RTX - 1) / RTX, by = (g.nn[1] + RTY - 1) / RTY, bz = (g.nn[2] + zc - 1) / zc;
  return bx * by * bz;
}

template <typename T, bool MIX, int SCHEME, bool FS>
static size_t residual_smem() {
  constexpr int NIP = (SCHEME == SCHEME_TETRA2) ? 2 : 1;
  return 2 * MAX_PHASE * 8 + 2 * (RTX * RTY / 32) * 8 + 2 * VY * VX * sizeof(VoxV<T, NIP, FS ? 9 : 6>) +
         2 * 3 * NY2 * NX2 * sizeof(NodeV<MIX>) + 2 * 3 * NY2 * NX2 * sizeof(T);
}

template <typename T, bool MIX, int SCHEME, bool FS>
static int launch_res_impl(const ResidualArgs& a, cudaStream_t s) {
  dim3 blk(RTX, RTY);
  const int zc = residual_zchunk(a.g);
  dim3 grd((a.g.nn[0] + RTX - 1) / RTX, (a.g.nn[1] + RTY - 1) / RTY, (a.g.nn[2] + zc - 1) / zc);
  ResidualArgs aa = a;
  aa.zchunk = zc;
  size_t sm = residual_smem<T, MIX, SCHEME, FS>();
  static bool attr_set = false;   // per template instance; the attribute is per function
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_residual<T, MIX, SCHEME, FS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  k_residual<T, MIX, SCHEME, FS><<<grd, blk, sm, s>>>(aa);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_residual(const ResidualArgs& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    return launch_residual_f32(a, s);   // thread-per-node FP32 kernel (k_residual_f32.cu)
  } else {
    const bool fs = a.g.finite_strain != 0;
    if (a.g.scheme == SCHEME_TETRA2)
      return fs ? launch_res_impl<T, false, SCHEME_TETRA2, true>(a, s) : launch_res_impl<T, false, SCHEME_TETRA2, false>(a, s);
    return fs ? launch_res_impl<T, false, SCHEME_HEX1, true>(a, s) : launch_res_impl<T, false, SCHEME_HEX1, false>(a, s);
  }
}

template int launch_residual<double>(const ResidualArgs&, cudaStream_t);
template int launch_residual<float>(const ResidualArgs&, cudaStream_t);

}  // namespace dtt

// Stress / divergence / reference-operator kernel of the mixed path (same operator as
// k_residual.cu: Eq. 3 with the HEX1 / TETRA2 gradients of Section 3.1.1, the Paux
// reference medium of Section 3.2.3 and the symmetry weights W of Table 1), organised for
// instruction throughput on B300:
//
//  * a CTA owns a 32 x 8 tile of node columns (the last x tile 33 x 8 when x is not
//    periodic and has 32 k + 1 nodes, rather than a tile of one column) and marches along
//    z one voxel layer at a time; the layer between node planes L and L+1 is processed in
//    two phases:
//      A. one thread per voxel of the 33 x 9 halo layer forms, once, the gradients of its
//         points, the stress sigma = C:(eps* + sym grad u~) and, on the layers that need
//         it, the reference-medium flux tau_cd = (2 mu0 + lambda0 delta_cd) d(.)_c/dx_d,
//         and stores them in shared memory (structure of arrays);
//      B. one thread per node gathers, from the 4 voxels of the layer around its column,
//         the divergence contributions to node L (as their lower corner) and to node L+1
//         (as their upper corner); node L is then complete and its outputs are written;
//  * u~ sits in shared memory as interleaved (hi, lo) pairs, so that one 64-bit load
//    fetches a corner and one packed subtraction forms both halves of a difference;
//  * TETRA2: the two tetrahedra of a voxel are the two lanes of packed FP32x2 arithmetic
//    (gradients, stress, flux, the stored point data); in phase B a voxel's lane pair
//    feeds node L from one tetrahedron and node L+1 from the other, so each gather is
//    one packed FMA per stress value;
//  * u~, the step Delta and the voxel phases of node planes sit in a 4-slot ring filled
//    with cp.async two planes ahead (layer L reads planes L and L+1 while L+2 and L+3
//    are in flight); the phases travel as aligned 4-byte words where the grid allows;
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

#include <map>
#include <mutex>
#include <queue>
#include <tuple>
#include <vector>

namespace dtt {

namespace {

constexpr int FTX = 32, FTY = 8;
constexpr int FVX = FTX + 1, FVY = FTY + 1;
constexpr int NVL = FVX * FVY;                   // 297 voxels per layer
constexpr int FTHREADS = 320;
constexpr int FHX = FTX + 2, FHY = FTY + 2;
constexpr int FPL = FHY * FHX;                   // 340 positions per node plane
constexpr int RING = 4;                         // node-plane ring slots
constexpr int PWX = 40;                         // phase bytes per voxel row in word mode
template <bool FS> struct PointLayout {
  static constexpr int NS = FS ? 9 : 6;          // stress values per point (Pi or sigma); the flux adds 9
};

__device__ __forceinline__ void cp_async4(void* smem_ptr, const void* gptr) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gptr));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ int wrapi(int i, int n, int per) {
  if (per) { i %= n; if (i < 0) i += n; return i; }
  return (i < 0 || i >= n) ? -1 : i;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{ .reg .b64 ra, rb, rr; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; sub.rn.f32x2 rr, ra, rb; mov.b64 {%0, %1}, rr; }"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
// (ph + pl) - (qh + ql) of float-float pairs, formed from their differences
__device__ __forceinline__ float fd(float2 p, float2 q) {
  const float2 d = sub2(p, q);
  return __fadd_rn(d.x, d.y);
}

// compensated FP32 accumulators, two lanes at once (TwoSum per lane)
struct Acc2x2 {
  float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 x) {
    const float2 t = add2(s, x);
    const float2 z = sub2(t, s);
    c = add2(c, add2(sub2(s, sub2(t, z)), sub2(x, z)));
    s = t;
  }
  __device__ __forceinline__ double value(int lane) const {
    return lane ? (double)s.y + (double)c.y : (double)s.x + (double)c.x;
  }
};

// reference flux tau = R0 : grad u of both points at once (Paux or isotropic medium)
__device__ __forceinline__ float2 ref_flux2(const float2 (&Gm)[3][3], int c, int d, float lam0, float mu0, bool iso) {
  if (iso) {
    float2 v = mul2(bc2(mu0), add2(Gm[c][d], Gm[d][c]));
    if (c == d) v = fma2(bc2(lam0), add2(add2(Gm[0][0], Gm[1][1]), Gm[2][2]), v);
    return v;
  }
  return mul2(bc2(2.f * mu0 + (c == d ? lam0 : 0.f)), Gm[c][d]);
}
__device__ __forceinline__ float ref_flux1(const float (&Gm)[3][3], int c, int d, float lam0, float mu0, bool iso) {
  if (iso) return (c == d ? lam0 * (Gm[0][0] + Gm[1][1] + Gm[2][2]) : 0.f) + mu0 * (Gm[c][d] + Gm[d][c]);
  return (2.f * mu0 + (c == d ? lam0 : 0.f)) * Gm[c][d];
}

}  // namespace

// PHW: voxel phases loaded as aligned 4-byte words (x extent a multiple of 4, x not
// periodic, phase array 4-byte aligned); otherwise one byte per halo position.
// PART (exact Anderson mode, whose R_{i-1} = p_i + A0 c needs the reference flux only next
// to the constrained nodes): 0 = one pass doing everything; 1 = the pass without the flux
// (no Delta ring, no flux point data: less shared memory and fewer registers), which leaves
// R and the Gram row of the node planes tile_z +- 1 to PART 2; 2 = one CTA per marked xy
// tile over those planes only, writing their R and Gram row (partials after the chunks').
template <int SCHEME, bool FS, bool PHW, int PART>
__global__ void __launch_bounds__(FTHREADS, 2)
k_residual_f32(ResidualArgs a) {
  constexpr bool TET = SCHEME == SCHEME_TETRA2;
  constexpr int NS = PointLayout<FS>::NS;
  constexpr int NPT = TET ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sU = (float2*)smem_raw;                       // [RING][3][FPL] u~ (hi, lo)
  float* sD = (float*)(sU + RING * 3 * FPL);            // [RING][3][FPL] Delta (not in PART 1)
  float* sSf = PART == 1 ? sD : sD + RING * 3 * FPL;    // stress point data [NS][NVL] (x NPT floats)
  float* sTf = sSf + NS * NVL * NPT;                    // flux point data [9][NVL] (x NPT floats; not in PART 1)
  uint8_t* sP = PART == 1 ? (uint8_t*)sTf : (uint8_t*)(sTf + 9 * NVL * NPT);   // phases: [RING][FPL] bytes, or [RING][FVY][PWX] words
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
  const long long NN = g.nnodes;
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];
  int z0 = blockIdx.z * zc;
  int z1 = min(z0 + zc, nnz);
  const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
  // without a PART 2 launch, the chunk CTAs of the lowest chunk zero its partials slots
  if (PART != 2 && a.split != 1 && blockIdx.z == 0 && tid < RES_STRIDE)
    a.partials[(long long)RES_STRIDE * ((long long)gridDim.x * gridDim.y * gridDim.z + blockIdx.x +
                                        (long long)gridDim.x * blockIdx.y) + tid] = 0.0;

  float* po = (float*)a.pout;
  float* xo = nullptr;
  float* ro = nullptr;
  const float* gprev = nullptr;
  const float* dfield = nullptr;
  const float* Rq[3] = {nullptr, nullptr, nullptr};   // the other three R slots, (rslot + 1 + k) % 4
  int rslot = -1;
  bool tau_on = true, tau_from_delta = false;
  int tz_lo = -(1 << 29), tz_hi = 1 << 29;
  int fl_lo = 1 << 30, fl_hi = -(1 << 30);   // PART 1: node planes whose R and Gram row PART 2 forms
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
      for (int k = 0; k < 3; ++k) Rq[k] = (const float*)a.rring[(rslot + 1 + k) % 4];
      if (a.exact) {
        gprev = nullptr;
        const int2 zr = a.tile_z[blockIdx.y * gridDim.x + blockIdx.x];
        if (PART == 2 && zr.x <= zr.y) {
          z0 = max(zr.x - 1, 0);
          z1 = min(zr.y + 2, nnz);
        }
        tau_on = zr.x <= zr.y && zr.y >= z0 - 1 && zr.x <= z1;
        if (!tau_on) dfield = nullptr;
        tz_lo = zr.x;
        tz_hi = zr.y;
        if (PART == 1 && zr.x <= zr.y) {
          fl_lo = zr.x - 1;
          fl_hi = zr.y + 1;
        }
      }
    } else {
      tau_on = false;
    }
  } else {
    tau_on = false;
  }
  if (PART == 2 && !(ro && tau_on)) {   // no flux node planes in this tile (or no R yet)
    if (tid < RES_STRIDE) a.partials[RES_STRIDE * blk + tid] = 0.0;
    return;
  }
  if (PART == 1) {
    tau_on = false;
    dfield = nullptr;
  }
  const float lam0 = a.f_lam0, mu0 = a.f_mu0;
  const bool iso = g.ref_iso != 0;
  const float inv2h = a.f_inv2h, inv4h = a.f_inv4h;
  const float c4h = inv4h;
  const float (&eps)[3][3] = a.f_eps;

  // ---- phase words: 10 aligned words per voxel row cover voxels x0 - 4 .. x0 + 35
  int w_off = -1;                  // byte offset of this thread's word in a voxel plane, -1: none
  if (PHW && tid < FVY * (PWX / 4)) {
    const int ly = tid / (PWX / 4), xs = x0 - 4 + 4 * (tid % (PWX / 4));
    const int vy = wrapi(y0 - 1 + ly, g.nvox[1], g.periodic[1]);
    if (vy >= 0 && xs >= 0 && xs + 4 <= g.nvox[0]) w_off = xs + g.nvox[0] * vy;
  }
  // ---- plane loader (each thread owns at most two of the 34 x 10 positions)
  // position m of this thread: q = tid + m * FTHREADS (m = 1 only for the first FPL - FTHREADS threads)
  const int nq = tid + FTHREADS < FPL ? 2 : 1;
  int q_node[2] = {-1, -1}, q_vox[2] = {-1, -1};     // in-plane indices (a plane holds < 2^31 nodes)
  for (int m = 0; m < nq; ++m) {
    const int q = tid + m * FTHREADS;
    const int lx = q % FHX, ly = q / FHX;
    const int gi = wrapi(x0 - 1 + lx, nnx, g.periodic[0]);
    const int gj = wrapi(y0 - 1 + ly, nny, g.periodic[1]);
    q_node[m] = (gi >= 0 && gj >= 0) ? gi + nnx * gj : -1;
    const int vx = wrapi(x0 - 1 + lx, g.nvox[0], g.periodic[0]);
    const int vy = wrapi(y0 - 1 + ly, g.nvox[1], g.periodic[1]);
    q_vox[m] = (vx >= 0 && vy >= 0) ? vx + g.nvox[0] * vy : -1;
  }
  const long long plane_n = (long long)nnx * nny, plane_v = (long long)g.nvox[0] * g.nvox[1];
  auto load_plane = [&](int kk) {
    const int slot = kk & (RING - 1);
    const int kw = wrapi(kk, nnz, g.periodic[2]);
    const int vz = wrapi(kk, g.nvox[2], g.periodic[2]);
    // Delta is read only on planes next to the layers that carry the flux
    const bool dplane = dfield && kk >= tz_lo - 1 && kk <= tz_hi + 1;
    #pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m >= nq) break;
      const bool ok = kw >= 0 && q_node[m] >= 0;
      const long long n = ok ? q_node[m] + plane_n * kw : 0;
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int si = (slot * 3 + c) * FPL + (tid + m * FTHREADS);
        if (ok) {
          cp_async4(&sU[si].x, a.uhi + c * NN + n);
          cp_async4(&sU[si].y, a.ulo + c * NN + n);
          if (dplane) cp_async4(&sD[si], dfield + c * NN + n);
        } else {
          sU[si] = make_float2(0.f, 0.f);
          if (dplane) sD[si] = 0.f;
        }
      }
      if (!PHW) {
        uint8_t ph = 255;   // 255 = no voxel
        if (vz >= 0 && q_vox[m] >= 0) ph = a.phase[q_vox[m] + plane_v * vz];
        sP[slot * FPL + (tid + m * FTHREADS)] = ph;
      }
    }
    if (PHW && tid < FVY * (PWX / 4)) {
      uint32_t* dst = (uint32_t*)(sP + slot * FVY * PWX) + tid;
      if (vz >= 0 && w_off >= 0) cp_async4(dst, a.phase + w_off + plane_v * vz);
      else *dst = 0xffffffffu;
    }
  };

  Acc2x2 acc_sp;            // lanes: sum w sigma:sigma, sum p^2
  Acc2x2 acc_g01, acc_g23;  // Gram row: lanes (R slot rslot, slot rslot + 1), (rslot + 2, rslot + 3)

  // the wide last x tile: threads FTX FTY .. + FTY - 1 (idle in phase B otherwise) own the
  // final node column, tx = FTX
  const bool xtra = tid >= FTX * FTY && tid < FTX * FTY + FTY && blockIdx.x == gridDim.x - 1 && res_wide_last_x(g, FTX);
  const bool node_thread = tid < FTX * FTY || xtra;
  const int tx = xtra ? FTX : tid % FTX, ty = xtra ? tid - FTX * FTY : tid / FTX;
  const int i = x0 + tx, j = y0 + ty;
  const bool active = node_thread && (i < nnx && j < nny);
  const bool vox_thread = tid < NVL;
  const int vlx = tid < FTX * FVY ? (tid % FTX) : FTX;
  const int vly = tid < FTX * FVY ? (tid / FTX) : (tid - FTX * FVY);
  const int vslot = vly * FVX + vlx;
  const bool own_xy = vlx >= 1 && vly >= 1 && (x0 - 1 + vlx) < g.nvox[0] && (y0 - 1 + vly) < g.nvox[1];

  // x / y faces of this thread's node column: DOF flags and Neumann weights per component
  // bits 3c: (node, c) is not a DOF; bits 3c+1..3c+2: number of Neumann faces through it
  int fxy = 0;
  {
    const int idx[2] = {i, j};
    #pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (g.periodic[d]) continue;
      int f = -1;
      if (idx[d] == 0) f = 0;
      else if (idx[d] == g.nn[d] - 1) f = 1;
      if (f < 0) continue;
      #pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int t = g.bc[d][f][c];
        if (t == BC_D) fxy |= 1 << (3 * c);
        else if (t == BC_N) fxy += 2 << (3 * c);
      }
    }
  }

  float Fc[3] = {0.f, 0.f, 0.f}, F0c[3] = {0.f, 0.f, 0.f};

  // ring of RING node planes (slot = plane & 3), filled two planes ahead: layer L reads
  // planes L and L+1 while L+2 and L+3 are in flight
  load_plane(z0 - 1);
  load_plane(z0);
  cp_async_commit();
  if (z0 + 1 <= z1) load_plane(z0 + 1);
  cp_async_commit();
  cp_async_wait_1();
  __syncthreads();

  long long nL = (long long)i + (long long)nnx * (j + (long long)nny * (z0 - 1));
  for (int L = z0 - 1; L < z1; ++L, nL += plane_n) {
    if (L + 3 <= z1) load_plane(L + 3);
    cp_async_commit();
    const int s0 = L & (RING - 1), s1 = (L + 1) & (RING - 1);

    uint8_t cm = 0;
    float pg[3] = {0.f, 0.f, 0.f}, pr[3][3];
    const bool fin = active && L >= z0;
    if (fin) {
      cm = a.cmask ? a.cmask[nL] : 0;
      if (ro) {
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (gprev) pg[c] = gprev[c * NN + nL];
          #pragma unroll
          for (int k = 0; k < 3; ++k) pr[k][c] = Rq[k][c * NN + nL];
        }
      }
    }

    const bool tau_L = tau_on && L >= tz_lo - 1 && L <= tz_hi;
    const bool need_gd = tau_L && tau_from_delta;
    // ---------------- phase A: point data of voxel layer L
    if (vox_thread) {
      const uint8_t ph = PHW ? sP[s0 * FVY * PWX + vly * PWX + vlx + 3] : sP[s0 * FPL + vly * FHX + vlx];
      if (ph == 255) {
        if constexpr (TET) {
          #pragma unroll
          for (int q = 0; q < NS; ++q) ((float2*)sSf)[q * NVL + vslot] = make_float2(0.f, 0.f);
          if (tau_L) {
            #pragma unroll
            for (int q = 0; q < 9; ++q) ((float2*)sTf)[q * NVL + vslot] = make_float2(0.f, 0.f);
          }
        } else {
          #pragma unroll
          for (int q = 0; q < NS; ++q) sSf[q * NVL + vslot] = 0.f;
          if (tau_L) {
            #pragma unroll
            for (int q = 0; q < 9; ++q) sTf[q * NVL + vslot] = 0.f;
          }
        }
      } else {
        const float lam = sLam[ph], mu = sMu[ph];
        const bool own = PART != 2 && own_xy && L >= z0 && L < g.nvox[2];
        const float2* U0 = sU + s0 * 3 * FPL + vly * FHX + vlx;
        const float2* U1 = sU + s1 * 3 * FPL + vly * FHX + vlx;
        const float* D0 = sD + s0 * 3 * FPL + vly * FHX + vlx;
        const float* D1 = sD + s1 * 3 * FPL + vly * FHX + vlx;
        // corner b = cx + 2 cy + 4 cz of the voxel, component c
        auto cu = [&](int b, int c) { return ((b >> 2) ? U1 : U0)[c * FPL + ((b >> 1) & 1) * FHX + (b & 1)]; };
        auto cd = [&](int b, int c) { return ((b >> 2) ? D1 : D0)[c * FPL + ((b >> 1) & 1) * FHX + (b & 1)]; };
        if constexpr (TET) {
          // lanes (T1, T2): T1 = corners {0, 3, 5, 6}, T2 = {1, 2, 4, 7} as (a, b, c, e);
          // with X = (b-a | a-b) and Y = (c-e | e-c):
          //   d/dx = X + Y,  d/dy = (X - Y) * (1 | -1),  d/dz = (c-a) + (e-b)   (all / 2h)
          const float2 i2 = bc2(inv2h), i2m = make_float2(inv2h, -inv2h);
          auto grad_u = [&](float2 (&G)[3][3]) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 u0 = cu(0, c), u1 = cu(1, c), u2 = cu(2, c), u3 = cu(3, c);
              const float2 u4 = cu(4, c), u5 = cu(5, c), u6 = cu(6, c), u7 = cu(7, c);
              const float2 dca = make_float2(fd(u5, u0), fd(u4, u1));
              const float2 deb = make_float2(fd(u6, u3), fd(u7, u2));
              const float2 X = make_float2(fd(u3, u0), fd(u1, u2));
              const float2 Y = make_float2(fd(u5, u6), fd(u7, u4));
              G[c][2] = mul2(add2(dca, deb), i2);
              G[c][0] = mul2(add2(X, Y), i2);
              G[c][1] = mul2(sub2(X, Y), i2m);
            }
          };
          auto grad_d = [&](float2 (&G)[3][3]) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float v0 = cd(0, c), v1 = cd(1, c), v2 = cd(2, c), v3 = cd(3, c);
              const float v4 = cd(4, c), v5 = cd(5, c), v6 = cd(6, c), v7 = cd(7, c);
              const float2 gca = sub2(make_float2(v5, v4), make_float2(v0, v1));
              const float2 geb = sub2(make_float2(v6, v7), make_float2(v3, v2));
              const float2 gX = sub2(make_float2(v3, v1), make_float2(v0, v2));
              const float2 gY = sub2(make_float2(v5, v7), make_float2(v6, v4));
              G[c][2] = mul2(add2(gca, geb), i2);
              G[c][0] = mul2(add2(gX, gY), i2);
              G[c][1] = mul2(sub2(gX, gY), i2m);
            }
          };
          float2 G[3][3];
          grad_u(G);
          float2* o = (float2*)sSf + vslot;
          float2* ot = (float2*)sTf + vslot;
          if constexpr (FS) {
            float2 H[3][3], S[3][3];
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int d = 0; d < 3; ++d) H[c][d] = add2(bc2(eps[c][d]), G[c][d]);
            #pragma unroll
            for (int p = 0; p < 3; ++p)
              #pragma unroll
              for (int q = p; q < 3; ++q) {
                float2 v = add2(H[p][q], H[q][p]);
                #pragma unroll
                for (int k = 0; k < 3; ++k) v = fma2(H[k][p], H[k][q], v);
                S[p][q] = S[q][p] = mul2(bc2(0.5f), v);
              }
            const float2 tr = add2(add2(S[0][0], S[1][1]), S[2][2]);
            const float2 ltr = mul2(bc2(lam), tr);
            #pragma unroll
            for (int p = 0; p < 3; ++p)
              #pragma unroll
              for (int q = p; q < 3; ++q) {
                const float2 v = mul2(bc2(2.f * mu), S[p][q]);
                S[p][q] = S[q][p] = (p == q) ? add2(v, ltr) : v;
              }
            float2 s2v = make_float2(0.f, 0.f);
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int d = 0; d < 3; ++d) {
                float2 v = S[c][d];
                #pragma unroll
                for (int k = 0; k < 3; ++k) v = fma2(H[c][k], S[k][d], v);
                o[(3 * c + d) * NVL] = v;
                s2v = fma2(v, v, s2v);
              }
            if (own) acc_sp.add(make_float2(0.5f * (s2v.x + s2v.y), 0.f));
          } else {
            const float2 exx = add2(bc2(eps[0][0]), G[0][0]), eyy = add2(bc2(eps[1][1]), G[1][1]);
            const float2 ezz = add2(bc2(eps[2][2]), G[2][2]);
            const float2 eyz = fma2(bc2(0.5f), add2(G[1][2], G[2][1]), bc2(eps[1][2]));
            const float2 exz = fma2(bc2(0.5f), add2(G[0][2], G[2][0]), bc2(eps[0][2]));
            const float2 exy = fma2(bc2(0.5f), add2(G[0][1], G[1][0]), bc2(eps[0][1]));
            const float2 ltr = mul2(bc2(lam), add2(add2(exx, eyy), ezz));
            const float2 m2 = bc2(2.f * mu);
            const float2 sxx = fma2(m2, exx, ltr), syy = fma2(m2, eyy, ltr), szz = fma2(m2, ezz, ltr);
            const float2 syz = mul2(m2, eyz), sxz = mul2(m2, exz), sxy = mul2(m2, exy);
            o[0 * NVL] = sxx;
            o[1 * NVL] = syy;
            o[2 * NVL] = szz;
            o[3 * NVL] = syz;
            o[4 * NVL] = sxz;
            o[5 * NVL] = sxy;
            if (own) {
              const float2 dg = fma2(szz, szz, fma2(syy, syy, mul2(sxx, sxx)));
              const float2 od = fma2(sxy, sxy, fma2(sxz, sxz, mul2(syz, syz)));
              const float2 s2v = fma2(bc2(2.f), od, dg);
              acc_sp.add(make_float2(0.5f * (s2v.x + s2v.y), 0.f));
            }
          }
          if (tau_L) {
            // reference flux (few layers): the gradient of Delta, or of u~ again
            float2 T[3][3];
            if (tau_from_delta) grad_d(T);
            else grad_u(T);
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int d = 0; d < 3; ++d) ot[(3 * c + d) * NVL] = ref_flux2(T, c, d, lam0, mu0, iso);
          }
        } else {
          // HEX1: one point at the voxel centre
          float G[3][3], GD[3][3];
          #pragma unroll
          for (int c = 0; c < 3; ++c) {
            float2 u[8];
            #pragma unroll
            for (int b = 0; b < 8; ++b) u[b] = cu(b, c);
            auto d = [&](int p, int q) { return fd(u[p], u[q]); };
            G[c][0] = (d(1, 0) + d(3, 2) + d(5, 4) + d(7, 6)) * inv4h;
            G[c][1] = (d(2, 0) + d(3, 1) + d(6, 4) + d(7, 5)) * inv4h;
            G[c][2] = (d(4, 0) + d(5, 1) + d(6, 2) + d(7, 3)) * inv4h;
            if (need_gd) {
              float ud[8];
              #pragma unroll
              for (int b = 0; b < 8; ++b) ud[b] = cd(b, c);
              GD[c][0] = ((ud[1] - ud[0]) + (ud[3] - ud[2]) + (ud[5] - ud[4]) + (ud[7] - ud[6])) * inv4h;
              GD[c][1] = ((ud[2] - ud[0]) + (ud[3] - ud[1]) + (ud[6] - ud[4]) + (ud[7] - ud[5])) * inv4h;
              GD[c][2] = ((ud[4] - ud[0]) + (ud[5] - ud[1]) + (ud[6] - ud[2]) + (ud[7] - ud[3])) * inv4h;
            }
          }
          float* o = sSf + vslot;
          float* ot = sTf + vslot;
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
                S[p][q] = S[q][p] = 0.5f * v;
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
            if (own) acc_sp.add(make_float2(s2, 0.f));
          } else {
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
            if (own) acc_sp.add(make_float2(sxx * sxx + syy * syy + szz * szz + 2.f * (syz * syz + sxz * sxz + sxy * sxy), 0.f));
          }
          if (tau_L) {
            #pragma unroll
            for (int c = 0; c < 3; ++c)
              #pragma unroll
              for (int dd = 0; dd < 3; ++dd)
                ot[(3 * c + dd) * NVL] =
                    tau_from_delta ? ref_flux1(GD, c, dd, lam0, mu0, iso) : ref_flux1(G, c, dd, lam0, mu0, iso);
          }
        }
      }
    }
    cp_async_wait_1();   // plane L+2 has landed (L+3 may still be in flight)
    __syncthreads();

    // ---------------- phase B: gather into node L (lower corner) and node L+1 (upper corner)
    float Fn[3] = {0.f, 0.f, 0.f}, F0n[3] = {0.f, 0.f, 0.f};
    if (active) {
      if constexpr (TET) {
        // voxels whose lower-corner point is T1 accumulate into A = (node L | node L+1),
        // the others into B = (node L+1 | node L)
        float2 A[3], B[3], A0[3], B0[3];
        #pragma unroll
        for (int c = 0; c < 3; ++c) A[c] = B[c] = A0[c] = B0[c] = make_float2(0.f, 0.f);
        #pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
          #pragma unroll
          for (int ex = 0; ex < 2; ++ex) {
            if (ex == 1 && tx == FTX) continue;   // right of the final column: no voxel
            const int v = (ty + ey) * FVX + (tx + ex);
            const int dx = 1 - ex, dy = 1 - ey;
            const bool tlo = (dx + dy) & 1;
            const float2 SX = bc2(dx ? 1.f : -1.f), SY = bc2(dy ? 1.f : -1.f);
            const float2 SZ = tlo ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f);
            const float2* q = (const float2*)sSf + v;
            const float2* qt = (const float2*)sTf + v;
            auto gather = [&](float2 (&F)[3], float2 (&F0)[3]) {
              if constexpr (FS) {
                #pragma unroll
                for (int c = 0; c < 3; ++c)
                  F[c] = fma2(q[(3 * c + 2) * NVL], SZ, fma2(q[(3 * c + 1) * NVL], SY, fma2(q[(3 * c) * NVL], SX, F[c])));
              } else {
                const float2 sxx = q[0], syy = q[NVL], szz = q[2 * NVL];
                const float2 syz = q[3 * NVL], sxz = q[4 * NVL], sxy = q[5 * NVL];
                F[0] = fma2(sxz, SZ, fma2(sxy, SY, fma2(sxx, SX, F[0])));
                F[1] = fma2(syz, SZ, fma2(syy, SY, fma2(sxy, SX, F[1])));
                F[2] = fma2(szz, SZ, fma2(syz, SY, fma2(sxz, SX, F[2])));
              }
              if (tau_L) {
                #pragma unroll
                for (int c = 0; c < 3; ++c)
                  F0[c] = fma2(qt[(2 + 3 * c) * NVL], SZ,
                               fma2(qt[(1 + 3 * c) * NVL], SY, fma2(qt[(3 * c) * NVL], SX, F0[c])));
              }
            };
            if (tlo) gather(B, B0);
            else gather(A, A0);
          }
        }
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          Fc[c] += A[c].x + B[c].y;
          Fn[c] = A[c].y + B[c].x;
          F0c[c] += A0[c].x + B0[c].y;
          F0n[c] = A0[c].y + B0[c].x;
        }
      } else {
        #pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
          #pragma unroll
          for (int ex = 0; ex < 2; ++ex) {
            if (ex == 1 && tx == FTX) continue;   // right of the final column: no voxel
            const int v = (ty + ey) * FVX + (tx + ex);
            const int dx = 1 - ex, dy = 1 - ey;
            const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f;
            const float* q = sSf + v;
            const float* qt = sTf + v;
            float t[3];
            if constexpr (FS) {
              #pragma unroll
              for (int c = 0; c < 3; ++c) t[c] = q[(3 * c) * NVL] * sx + q[(3 * c + 1) * NVL] * sy;
              #pragma unroll
              for (int c = 0; c < 3; ++c) {
                Fc[c] += t[c] - q[(3 * c + 2) * NVL];
                Fn[c] += t[c] + q[(3 * c + 2) * NVL];
              }
            } else {
              const float sxx = q[0], syy = q[NVL], szz = q[2 * NVL];
              const float syz = q[3 * NVL], sxz = q[4 * NVL], sxy = q[5 * NVL];
              t[0] = sxx * sx + sxy * sy;
              t[1] = sxy * sx + syy * sy;
              t[2] = sxz * sx + syz * sy;
              Fc[0] += t[0] - sxz; Fn[0] += t[0] + sxz;
              Fc[1] += t[1] - syz; Fn[1] += t[1] + syz;
              Fc[2] += t[2] - szz; Fn[2] += t[2] + szz;
            }
            if (tau_L) {
              #pragma unroll
              for (int c = 0; c < 3; ++c) {
                const float tt = qt[(3 * c) * NVL] * sx + qt[(1 + 3 * c) * NVL] * sy;
                F0c[c] += tt - qt[(2 + 3 * c) * NVL];
                F0n[c] += tt + qt[(2 + 3 * c) * NVL];
              }
            }
          }
        }
      }
      // node plane L is complete
      if (fin) {
        // z faces (uniform over the layer)
        int zf = -1;
        if (!g.periodic[2]) zf = (L == 0) ? 0 : (L == nnz - 1) ? 1 : -1;
        float p2loc = 0.f;
        float2 g01 = make_float2(0.f, 0.f), g23 = make_float2(0.f, 0.f);
        const bool fix_owned = PART == 1 && L >= fl_lo && L <= fl_hi;
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
          bool dof = !((fxy >> (3 * c)) & 1);
          float invW = (float)(1 << ((fxy >> (3 * c + 1)) & 3));
          if (zf >= 0) {
            const int t = g.bc[2][zf][c];
            if (t == BC_D) dof = false;
            else if (t == BC_N) invW *= 2.f;
          }
          float pv = 0.f, a0v = 0.f;
          if (dof) {
            pv = -Fc[c] * c4h * invW;
            if (tau_on) a0v = F0c[c] * c4h * invW;
          }
          const long long e = c * NN + nL;
          const bool free_dof = dof && !((cm >> c) & 1);
          if (free_dof) p2loc = fmaf(pv, pv, p2loc);
          if (PART != 2 && po) po[e] = pv;
          if (xo) xo[e] = pv + a0v;
          if (ro && !fix_owned) {
            const float rv = dof ? (pv - pg[c] + a0v) : 0.f;
            ro[e] = rv;
            if (free_dof) {
              const float2 r2 = bc2(rv);
              g01 = fma2(r2, make_float2(rv, pr[0][c]), g01);
              g23 = fma2(r2, make_float2(pr[1][c], pr[2][c]), g23);
            }
          }
        }
        if (PART != 2) acc_sp.add(make_float2(0.f, p2loc));
        if (ro && !fix_owned) {
          acc_g01.add(g01);
          acc_g23.add(g23);
        }
      }
    }
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
      Fc[c] = Fn[c];
      F0c[c] = F0n[c];
    }
    // the gather must finish before the next layer's phase A rewrites the point data
    __syncthreads();
  }
  cp_async_wait_all();

  // block reduction: compensated FP32 pairs across the warp, FP64 across warps
  Acc2x2 v3[3] = {acc_sp, acc_g01, acc_g23};
  const int warp = tid >> 5, lane = tid & 31;
  #pragma unroll
  for (int q = 0; q < 3; ++q) {
    Acc2x2 t = v3[q];
    #pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      float2 os, oc;
      os.x = __shfl_down_sync(0xffffffffu, t.s.x, off);
      os.y = __shfl_down_sync(0xffffffffu, t.s.y, off);
      oc.x = __shfl_down_sync(0xffffffffu, t.c.x, off);
      oc.y = __shfl_down_sync(0xffffffffu, t.c.y, off);
      t.add(os);
      t.c = add2(t.c, oc);
    }
    if (lane == 0) {
      // partial index: 0 sigma:sigma, 1 p^2, 2 + Gram slot
      const int rs = rslot < 0 ? 0 : rslot;
      const int i0 = q == 0 ? 0 : 2 + (rs + 2 * (q - 1)) % 4;
      const int i1 = q == 0 ? 1 : 2 + (rs + 2 * (q - 1) + 1) % 4;
      sRed[i0][warp] = t.value(0);
      sRed[i1][warp] = t.value(1);
    }
  }
  __syncthreads();
  if (tid < RES_STRIDE) {
    double t = 0.0;
    for (int w = 0; w < FTHREADS / 32; ++w) t += sRed[tid][w];
    a.partials[RES_STRIDE * blk + tid] = t;
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

// Modelled duration of the grid for a z chunk of zc planes: a CTA takes its chunk's voxel
// layers (planes + 1) plus a start-up cost of about 4 layers (ring fill, constants, block
// reduction); CTAs start in launch order (xy tiles, then z chunks) on the first free one of
// S resident slots.  (Fits the measured chunk sweeps on 256 x 256 x 128 and 384 x 384 x 192
// blocks to a few per cent.)
static double zchunk_makespan(int nnz, long long bxy, int zc, int S) {
  constexpr double C0 = 4.0;
  const long long full = bxy * (nnz / zc);
  const int rem = nnz % zc;
  const double d = zc + 1 + C0;
  // equal CTAs fill the slots round-robin: r slots end at (q + 1) d, the others at q d
  const long long q = full / S, r = full % S;
  std::priority_queue<double, std::vector<double>, std::greater<double>> slots;
  double end = 0.0;
  for (int k = 0; k < S; ++k) {
    const double t = (k < r ? q + 1 : q) * d;
    slots.push(t);
    end = std::max(end, t);
  }
  if (rem) {
    const double ds = rem + 1 + C0;
    for (long long k = 0; k < bxy; ++k) {
      const double t = slots.top() + ds;
      slots.pop();
      slots.push(t);
      end = std::max(end, t);
    }
  }
  return end;
}

// z planes per CTA: the chunk in [4, 64] with the shortest modelled duration (ties to the
// larger chunk), cached per grid shape.
int residual_f32_zchunk(const GridDev& g) {
  if (g.zc_override > 0) return g.zc_override;
  const long long bxy = (long long)res_ntx(g, FTX) * ((g.nn[1] + FTY - 1) / FTY);
  const int S = resident_ctas();
  const int nnz = g.nn[2];
  static std::mutex mu;
  static std::map<std::tuple<int, long long, int>, int> cache;
  const auto key = std::make_tuple(nnz, bxy, S);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int best = 64;
  double t_best = 1e300;
  for (int zc = 64; zc >= 4; --zc) {
    const double t = zchunk_makespan(nnz, bxy, zc, S);
    if (t < t_best * (1.0 - 1e-9)) {
      t_best = t;
      best = zc;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = best;
  return best;
}

int residual_f32_tile(int axis) { return axis == 0 ? FTX : FTY; }

// partials slots: one per chunk CTA, then one per xy tile (the flux-column pass)
int residual_f32_blocks(const GridDev& g) {
  int zc = residual_f32_zchunk(g);
  const int ntiles = res_ntx(g, FTX) * ((g.nn[1] + FTY - 1) / FTY);
  return ntiles * ((g.nn[2] + zc - 1) / zc) + ntiles;
}

template <int SCHEME, bool FS, int PART>
static int launch_part(const ResidualArgs& a, dim3 grd, size_t sm, bool phw, cudaStream_t s) {
  auto k = phw ? k_residual_f32<SCHEME, FS, true, PART> : k_residual_f32<SCHEME, FS, false, PART>;
  static bool attr[2] = {false, false};
  if (!attr[phw]) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    attr[phw] = true;
  }
  k<<<grd, FTHREADS, sm, s>>>(a);
  return (int)cudaGetLastError();
}

template <int SCHEME, bool FS>
static int launch_f32_impl(const ResidualArgs& a, cudaStream_t s) {
  const int zc = residual_f32_zchunk(a.g);
  dim3 grd(res_ntx(a.g, FTX), (a.g.nn[1] + FTY - 1) / FTY, (a.g.nn[2] + zc - 1) / zc);
  const long long nchunk = (long long)grd.x * grd.y * grd.z;
  ResidualArgs aa = a;
  aa.zchunk = zc;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) aa.f_eps[p][q] = (float)a.eps[p][q];
  aa.f_lam0 = (float)a.lam0;
  aa.f_mu0 = (float)a.mu0;
  aa.f_inv2h = (float)(1.0 / (2.0 * a.g.h));
  aa.f_inv4h = (float)(1.0 / (4.0 * a.g.h));
  constexpr int NPT = (SCHEME == SCHEME_TETRA2) ? 2 : 1;
  constexpr int NS = PointLayout<FS>::NS;
  // ring: u~ pairs (8 B) and Delta (4 B) per position; stress and flux point data; phases
  const size_t sm = (size_t)RING * 3 * FPL * (sizeof(float2) + sizeof(float)) +
                    (size_t)(NS + 9) * NVL * NPT * sizeof(float) + (size_t)RING * FVY * PWX;
  // the flux-free pass: no Delta ring and no flux point data
  const size_t sm_nf = (size_t)RING * 3 * FPL * sizeof(float2) + (size_t)NS * NVL * NPT * sizeof(float) +
                       (size_t)RING * FVY * PWX;
  static_assert(RING * FVY * PWX >= RING * FPL, "phase ring holds either layout");
  // word loads of the phases: every voxel row then starts on a 4-byte boundary
  const bool phw = a.g.nvox[0] % 4 == 0 && !a.g.periodic[0] && ((uintptr_t)a.phase & 3) == 0;
  const bool split = a.mode == 1 && a.exact && a.split != 0;
  if (!split) {
    aa.split = 0;
    return launch_part<SCHEME, FS, 0>(aa, grd, sm, phw, s);
  }
  int e = launch_part<SCHEME, FS, 1>(aa, grd, sm_nf, phw, s);
  if (e != 0 || a.split != 1) return e;
  ResidualArgs af = aa;
  af.partials = a.partials + RES_STRIDE * nchunk;
  return launch_part<SCHEME, FS, 2>(af, dim3(grd.x, grd.y, 1), sm, phw, s);
}

int launch_residual_f32(const ResidualArgs& a, cudaStream_t s) {
  const bool fs = a.g.finite_strain != 0;
  if (a.g.scheme == SCHEME_TETRA2)
    return fs ? launch_f32_impl<SCHEME_TETRA2, true>(a, s) : launch_f32_impl<SCHEME_TETRA2, false>(a, s);
  return fs ? launch_f32_impl<SCHEME_HEX1, true>(a, s) : launch_f32_impl<SCHEME_HEX1, false>(a, s);
}

}  // namespace dtt

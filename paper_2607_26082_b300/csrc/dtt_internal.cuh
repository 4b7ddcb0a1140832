// Internal declarations shared by the CUDA translation units of libdtt.
//
// Data layout in device memory (one grid):
//   * node arrays: component-major, x fastest: field[c * nnodes + i + nnx*(j + nny*k)],
//     nn_d = n_d + 1 on a non-periodic axis, n_d on a periodic one;
//   * u~ (the fluctuation displacement, Eq. 3): float64 in the FP64 path; in the mixed
//     path a float-float pair (hi, lo) so that differences of neighbouring values, and
//     thus strains, keep ~48 bits while every arithmetic operation stays in FP32;
//   * the other nodal fields (p, p~ ring, Anderson ring, spectra) are T = double (FP64
//     path) or float (mixed path);
//   * voxel phase ids: uint8, x fastest.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace dtt {

constexpr int BC_P = 0, BC_D = 1, BC_N = 2;
constexpr int T_DCT1 = 0, T_DCT3 = 1, T_DST1 = 2, T_DST3 = 3, T_DHT = 4;
constexpr int SCHEME_TETRA2 = 0, SCHEME_HEX1 = 1;
constexpr int MAX_PHASE = 256;
constexpr int HIST = 4096;

// Geometry passed by value to every kernel.
struct GridDev {
  int nvox[3];
  int nn[3];
  long long nnodes;
  double h;
  int scheme;
  int bc[3][2][3];  // [axis][face][component]
  int periodic[3];
  int zc_override;   // residual kernels: node planes per CTA (0: built-in choice)
  int fft_generic;   // 1: generic Stockham kernels for every length
  int finite_strain; // 1: first Piola-Kirchhoff stress (Section 5.2), 0: small strain
  int ref_iso;       // 1: isotropic reference medium (Section 3.2.3), 0: Paux
};

// Solver state kept on the device so that a whole iteration is a fixed sequence of
// launches (capturable in a CUDA graph) with no host decision in it.
struct Ctrl {
  int i_local;        // Anderson counter (reset to 0 when the contact zone changes)
  int iter;           // Green steps performed
  int done;           // 0 running, 1 converged, 2 iteration cap, 3 diverged (r not finite,
                      // r grown 1e6-fold, or the RMS of p grown 1e6-fold)
  int accel;          // accelerate at this iteration
  int max_iter;
  int acv_mod;
  int acv_on;         // 0 = u~, 1 = p~
  int contact_on;
  int update;         // contact-zone update at this iteration
  int changed;        // contact zone changed by the last update
  int n_updates;
  int n_accel;
  int n_vgap, n_vreact, n_mismatch, prev_valid;
  int hist_len;
  int no_stop;        // profiling: never stop on tolerance, cap or divergence
  int pslot;          // p-ring slot written by this iteration's residual kernel
  double tol, update_tol;
  double acv_pivot;
  double r, r0;
  double pn0;         // RMS of the projected p at the solve's first iterate
  double p2, s2;
  double alpha[4];
  float alpha_f[4];   // the same coefficients in FP32 (set with alpha; read by FP32 kernels)
  double gram[4][4];
  // Members above this line form the "head" that k_ctrl_residual_acv stages in shared
  // memory and accesses there; every member its control logic touches must stay above.
  double hist[HIST];
  unsigned int blocks_done;   // CTAs of the current k_proj_U that have finished (end of iteration)
};

// Sparse constraint rows (CSR over entries), disjoint supports.
struct RowsDev {
  int nrows;
  const int* ptr;        // nrows + 1
  const long long* dof;  // c * nnodes + node
  const double* a;
  const double* b;
  const double* target;  // value on u~ (U - A u*)
  double* mult;          // f_r = -lambda_r
  const double* ab;      // sum a b
  const double* aa;      // sum a a
};

struct ContactDev {
  int nnodes_face;
  const long long* node;   // flat node index of each surface node
  uint8_t* active;
  uint8_t* vgap;
  uint8_t* vreact;
  uint8_t* vgap_prev;
  uint8_t* vreact_prev;
  double* gap;
  double* fn;
  double* nvec;            // 3 x nnodes_face normals at the last evaluation
  double center[3];
  double radius;
};

// ---------------------------------------------------------------------------------
// Float-float helpers (mixed path).  TwoSum (Knuth) and Fast2Sum (Dekker): error-free
// transformations of a floating-point sum, written from their published definitions.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void ff_add(float& hi, float& lo, float d) {
  float s = __fadd_rn(hi, d);
  float bb = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  e = __fadd_rn(e, lo);
  float h2 = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(h2, s));
  hi = h2;
}
__device__ __forceinline__ void ff_set(float& hi, float& lo, double v) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}

// ---------------------------------------------------------------------------------
// Launch wrappers (kernels.cu).  T = double (FP64 path) or float (mixed path).
// ---------------------------------------------------------------------------------
struct ResidualArgs {
  GridDev g;
  const double* u64;
  const float* uhi;
  const float* ulo;
  const uint8_t* phase;
  const double* lam;
  const double* mu;
  int nphase;
  const uint8_t* cmask;   // bit c set: DOF (node, c) belongs to a row support / contact face
  double eps[3][3];
  double lam0, mu0;
  int mode;               // 0: p and p~ = p + A0 u~ ; 1: Anderson difference form ; 2: p only
  void* xout;             // mode 0: p~ (may be null)
  void* pout;             // modes 0, 2: p (may be null)
  const void* dfield;     // mode 1: Delta = last step of u~ (T); with `exact`, only the
                          // projections' correction of the last step
  // exact residual mode (mixed path, no null modes): the Green step inverts A0 exactly, so
  // R_{i-1} = p_i - g_{i-1} + A0 Delta_{i-1} = p_i + A0 c_{i-1} with c the projections'
  // correction (dfield); A0 c is formed only in CTAs whose node halo meets a row DOF or a
  // contact-face node: tile_z[ty * ntx + tx] = {zmin, zmax} of such nodes for the CTA's
  // xy tile (zmin > zmax: none)
  int exact;
  const int2* tile_z;
  // mixed kernel in the exact mode: 0 = one pass; 1 = a pass without the flux, then one CTA
  // per marked xy tile over the node planes tile_z +- 1 (short marked z ranges); 2 = the
  // pass without the flux alone (no marked tile)
  int split;
  void* pring[4];         // mode 1: p ring (slot i % 4)
  void* gring[4];         // mode 1: Green-input ring (g_{i-1} read from slot (i-1) % 4)
  void* rring[4];         // mode 1: Anderson residual ring (R_{i-1} into slot (i-1) % 4)
  double* partials;       // 2 per block: sum w sigma:sigma, sum p^2 (unmasked DOFs)
  const Ctrl* ctrl;       // if non-null: skip when done (mode 1 needs it)
  int zchunk;             // z planes per CTA (set by the launcher)
  // FP32 constants of the mixed kernel (set by its launcher from the fields above)
  float f_eps[3][3];
  float f_lam0, f_mu0, f_inv2h, f_inv4h;
};
// Residual partial sums: 6 doubles per CTA [w sigma:sigma, p^2, Gram 0..3] (the FP64
// kernel leaves the Gram entries 0; the FP32 kernel fills them in the Anderson mode).
constexpr int RES_STRIDE = 6;
// done flags of many grids' control blocks gathered into one array (batched solves)
int launch_batch_done(Ctrl* const* ctrls, int n, int* done, cudaStream_t s);
// condition kernel of the device-side solve loop (conditional WHILE node)
int launch_loop_continue(Ctrl* const* ctrls, const Ctrl* one, int n, cudaGraphConditionalHandle h, int* rounds,
                         int max_rounds, cudaStream_t s);
template <typename T> int launch_residual(const ResidualArgs& a, cudaStream_t s);
int residual_blocks(const GridDev& g);
int residual_zchunk(const GridDev& g);
int launch_residual_f32(const ResidualArgs& a, cudaStream_t s);
int residual_f32_blocks(const GridDev& g);
int residual_f32_tile(int axis);   // node tile of the mixed residual kernel along x (0) and y (1)
// xy tiles of the mixed residual kernel (tx x ty node columns).  When x is not periodic and
// holds tx k + 1 nodes, the last x tile also owns the final node column (tx + 1 wide), whose
// voxels to the right lie outside the grid, instead of a tile of one column.
__host__ __device__ inline bool res_wide_last_x(const GridDev& g, int tx) {
  return !g.periodic[0] && g.nn[0] > tx && g.nn[0] % tx == 1;
}
__host__ __device__ inline int res_ntx(const GridDev& g, int tx) {
  return res_wide_last_x(g, tx) ? g.nn[0] / tx : (g.nn[0] + tx - 1) / tx;
}
__host__ __device__ inline int res_tile_of_x(const GridDev& g, int i, int tx) {
  const int t = i / tx, n = res_ntx(g, tx);
  return t < n ? t : n - 1;
}
template <typename T> int residual_nblocks(const GridDev& g) {
  return sizeof(T) == 4 ? residual_f32_blocks(g) : residual_blocks(g);
}

// FFT route of one axis (shared by the three components: same length, per-component type).
struct FftAxisInfo {
  int use;                 // 1: FFT route; 0: dense contraction
  int L;                   // FFT length (2n, or n on a periodic axis)
  int nst;                 // number of Stockham stages
  int radix[12];
  const void* tw;          // L complex twiddles e^{-2 pi i m / L} (field precision)
  const void* ph;          // 2n complex e^{-i pi j / 2n} (quarter-wave types)
  const void* tw1;         // mixed path, L = 32 R: [R][32] float2 e^{-2 pi i l k1 / L} (warp passes)
};
struct FftParams {
  int axis, n, nn, L, nst;
  int radix[12];
  const void* tw;
  const void* ph;
  int type[3];
  int inverse;
  double scale;
  int comp0;
  int nnx, nny;
  long long npencil, NN;
  float fscale;            // scale in FP32 (mixed path)
  float finv_n;            // inv_n in FP32 (mixed path; no per-thread conversion)
  int generic;             // 1: generic Stockham kernels only (tuning choice)
  double inv_n;            // 1 / n (quarter-wave inverses)
  int incr;                // inverse x pass: add the result to u~ and store it as the step
  double* u64;
  float* uhi;
  float* ulo;
  void* step;
};
template <typename T>
int launch_fft_axis(const T* in, T* out, const FftParams& p, int ncomp, const Ctrl* ctrl, void* const* in_ring,
                    cudaStream_t s);
struct GreenTables;
template <typename T>
int launch_fft_z_green(const T* in, T* out, const FftParams& p, const GreenTables& gt, double lam0, double mu0,
                       int scheme, double h, int ncomp, const Ctrl* ctrl, cudaStream_t s);

// Isotropic reference medium: per-axis symbol factors shared by the three components
// (normal mixed conditions), the components present at each position, and the sign of
// the cross terms: sign[d] = +1 when the normal component's transform along axis d is a
// sine transform, -1 for a cosine transform; the (c, d) term carries sign[c] sign[d].
struct IsoTables {
  const double* s[3];
  const double* c[3];
  const float* sf[3];
  const float* cf[3];
  const uint8_t* valid[3];
  int sign[3];
  double null_thr;
};
// Tensor-core z pass (k_tensor_z.cu): per component, the active node rows [j0, j0 + nj)
// and spectral positions [k0, k0 + nk) of its z transform, the operand size P (a multiple
// of 32, >= nj and nk, the same for the three components), and the forward (P x P, rows =
// spectral positions) and inverse (rows = nodes) matrices packed chunk by chunk in the
// kernel's shared-memory operand layout, each chunk a TF32 high part and an FP32 remainder.
struct TzComp {
  const float* fwd;
  const float* inv;
  int j0, nj, k0, nk, P;
};
struct TzParams {
  TzComp c[3];
  int comp0;
  int nnx, nnz;
  long long npencil, NN, stride;
  unsigned int* err;       // set to 1 by a CTA whose bounded wait ran out
};

struct TransformTables {
  FftAxisInfo fft[3];
  int tz_use;              // 1: fused z pass as tensor-core contractions (mixed path)
  TzComp tz[3];
  unsigned int* tz_err;
  int types[3][3];         // [comp][axis]
  const void* fwd[3][3];   // [comp][axis] nn x nn row-major (spectral k, node j)
  const void* inv[3][3];   // [comp][axis] nn x nn row-major (node j, spectral k)
  const double* sin2q[3][3];   // sin^2(q_k / 2) at every spectral position (0 unused)
  const double* cos2q[3][3];   // cos^2(q_k / 2) (1 unused)
  const float* sin2q_f[3][3];  // the same tables in FP32
  const float* cos2q_f[3][3];
  double lam0, mu0;
  double null_thr[3];
  IsoTables iso;           // isotropic reference medium (GridDev::ref_iso)
};
struct GreenTables {
  const double* s[3][3];
  const double* cp[3][3];
  const float* sf[3][3];    // FP32 copies
  const float* cpf[3][3];
  double null_thr[3];
  float null_thr_f[3];
};
// symbol factor tables in the field precision (no conversions in the mixed path)
template <typename T>
__device__ __forceinline__ T gt_s(const GreenTables& gt, int c, int d, int k) {
  if constexpr (sizeof(T) == 4) return gt.sf[c][d][k];
  else return (T)gt.s[c][d][k];
}
template <typename T>
__device__ __forceinline__ T gt_c(const GreenTables& gt, int c, int d, int k) {
  if constexpr (sizeof(T) == 4) return gt.cpf[c][d][k];
  else return (T)gt.cp[c][d][k];
}
struct IncrTarget {
  double* u64;
  float* uhi;
  float* ulo;
  void* step;
};
// Warp-register passes of the mixed Green step (k_wfft.cu): one pass over rows along one
// axis; row r of outer index o of component c starts at c NN + o in_outer + r in_row; a
// transposed pass writes value k of that row to c NN + o out_outer + k out_k + r.
struct WfftPass {
  const float* in;
  void* const* in_ring;     // first pass: the Green input is ring slot i % 4
  float* out;
  int len, n, nrows;        // nodes along the axis, voxels along it, rows per outer index
  int rpt;                  // rows per CTA (even; set by the launcher)
  long long in_outer, in_row, out_outer, out_k, NN;
  int type[3];
  int inverse;
  float sc, inv_n;          // inverse scale 2/n (non-quarter types), 1/n (quarter-wave)
  const float2* tw1;
  const float2* ph;
  int comp0;
  float* uhi;               // last pass: u~ += result (float-float), step = result (if step)
  float* ulo;
  float* step;
};
int wfft_radix(int L);
bool wfft_supported(const GridDev& g, const TransformTables& tt);
int launch_wfft_green(const GridDev& g, const TransformTables& tt, const float* in, void* const* in_ring,
                      float* b1, float* b2, float* out, const IncrTarget* incr, int comp0, int ncomp,
                      const Ctrl* ctrl, cudaStream_t s, void (*mark)(int, cudaStream_t) = nullptr);
template <typename T>
int launch_transform_axis(const GridDev& g, const T* in, T* out, const TransformTables& tt,
                          int axis, int inverse, int ncomp_first, int ncomp, const Ctrl* ctrl,
                          cudaStream_t s, void* const* in_ring = nullptr, const IncrTarget* incr = nullptr);
// fused forward z DTT + Green multiply + inverse z DTT (FFT route on z only)
template <typename T>
int launch_z_green(const GridDev& g, const T* in, T* out, const TransformTables& tt, int ncomp_first, int ncomp,
                   const Ctrl* ctrl, cudaStream_t s);
// the same pass as two split-TF32 tensor-core contractions (mixed path, z operand <= 256)
int launch_tz_green(const float* in, float* out, const TzParams& p, const GreenTables& gt, double lam0, double mu0,
                    int scheme, double h, int ncomp, const Ctrl* ctrl, cudaStream_t s);
// rows [r0, r0 + nr) and columns [c0, c0 + ncol) of the nn x nn matrix M, packed for the
// tensor-core z pass with operand size P
void tz_pack_matrix(const double* M, int nn, int r0, int nr, int c0, int ncol, int P, std::vector<float>& out);
// Green step of the isotropic reference medium: a 3 x 3 solve per spectral position over
// the three components' spectra (component-major, node-grid positions), in place.
template <typename T>
int launch_green_iso(const GridDev& g, T* spec, const TransformTables& tt, const Ctrl* ctrl, cudaStream_t s);
template <typename T>
int launch_green_multiply(const GridDev& g, T* spec, const TransformTables& tt, int scheme,
                          const Ctrl* ctrl, cudaStream_t s);
template <typename T>
int launch_add_increment(const GridDev& g, const T* delta, double* u64, float* uhi, float* ulo,
                         T* step_out, const Ctrl* ctrl, cudaStream_t s);

// p: either p_direct, or (ring mode) p ring slot i % 4 with the same shifts applied to
// the Anderson residual slot (i-1) % 4 when i > 0.  With gram = 1 the kernel also adds the
// Gram-row contributions of its DOFs (partials: 5 per block [p^2, Gram 0..3]).
constexpr int PROJ_STRIDE = 5;
constexpr int CONT_STRIDE = 8;   // [p^2, n_vgap, n_vreact, mismatches, Gram 0..3]
template <typename T>
int launch_proj_P_rows(const GridDev& g, const RowsDev& r, T* p_direct, void* const* pring,
                       void* const* rring, int ring_mode, int gram, double* partials, const Ctrl* ctrl,
                       cudaStream_t s, T* step_clear = nullptr);
template <typename T>
int launch_proj_U_rows(const GridDev& g, const RowsDev& r, double* u64, float* uhi, float* ulo,
                       T* step, const Ctrl* ctrl, cudaStream_t s);
// The same projection, its last CTA also ending the iteration (the work of k_ctrl_end):
// one launch fewer per iteration when the rows' projection is the iteration's last step.
template <typename T>
int launch_proj_U_rows_end(const GridDev& g, const RowsDev& r, double* u64, float* uhi, float* ulo,
                           T* step, Ctrl* ctrl, cudaStream_t s);

struct ContactArgs {
  GridDev g;
  ContactDev c;
  const double* u64;
  const float* uhi;
  const float* ulo;
  double eps[3][3];
  const Ctrl* ctrl;
  double* partials;   // 3 per block: p^2, n_vgap, n_vreact (+ mismatches in [3])
  void* step_clear;   // exact residual mode: the step field, cleared at the face nodes (T)
};
template <typename T>
int launch_contact_eval(const ContactArgs& a, T* p_direct, void* const* pring, void* const* rring,
                        int ring_mode, int gram, cudaStream_t s);
int launch_contact_update(const ContactArgs& a, cudaStream_t s);
template <typename T>
int launch_contact_proj_U(const ContactArgs& a, double* u64, float* uhi, float* ulo, T* step,
                          cudaStream_t s);
int launch_contact_init(const ContactArgs& a, cudaStream_t s, int keep_active = 0);
int contact_blocks(int nface);

// Anderson on p~ in difference form: Gram row of R_{i-1}, then the accelerated Green input
//   g_i = sum_m alpha_m p_{i-3+m} - sum_{q<3} beta_q (R_k - p_{k+1} + g_k),  k = i-3+q,
//   beta_q = alpha_0 + ... + alpha_q   (g_i = p_i when not accelerating).
template <typename T>
int launch_acv_gram(const GridDev& g, void* const* rring, double* partials, const Ctrl* ctrl,
                    cudaStream_t s);
// gring: the ring of Green-input pointers read by the Green step (slot i % 4); gown: the
// grid's own Green-input buffers.  alias (FP32, exact residual mode only): an iteration
// without acceleration points gring[i % 4] at p_i's buffer instead of copying p_i, and an
// accelerated one reads the R ring only in the tiles of tile_z (the residual kernel's
// per-tile z ranges of constrained DOFs), where R_k and p_(k+1) can differ.
template <typename T>
int launch_acv_green_input(const GridDev& g, void* const* pring, void** gring, void* const* gown,
                           void* const* rring, const Ctrl* ctrl, int alias, const int2* tile_z, cudaStream_t s);
// Anderson on u~ (FP64 path): S ring of u~ copies, R = u~_i - S_{i-1}.
template <typename T>
int launch_acv_store(const GridDev& g, int acv_on, void* const* Sring, void* const* Rring,
                     const double* u64, double* partials, const Ctrl* ctrl, cudaStream_t s);
template <typename T>
int launch_acv_accel(const GridDev& g, int acv_on, void* const* Sring, void* const* Rring,
                     T* gbuf, double* u64, const Ctrl* ctrl, cudaStream_t s);
int acv_blocks(const GridDev& g);

// control kernels
int launch_ctrl_residual(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, const double* cp,
                         int ncont, double h, long long nnodes, long long nvox, cudaStream_t s);
int launch_ctrl_contact(Ctrl* c, cudaStream_t s);
int launch_ctrl_acv(Ctrl* c, const double* partials, int nblk, cudaStream_t s);
// Gram row from the fused sources: residual (RES_STRIDE, offset 2), projections
// (PROJ_STRIDE, offset 1), contact (CONT_STRIDE, offset 4)
int launch_ctrl_residual_acv(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, double h,
                             long long nnodes, long long nvox, cudaStream_t s);
int launch_ctrl_acv_fused(Ctrl* c, const double* rp, int nres, const double* pp, int nproj, const double* cp,
                          int ncont, cudaStream_t s);
int launch_ctrl_end(Ctrl* c, cudaStream_t s);

// utilities (k_util.cu)
int launch_to_double(long long n, const void* in, int in_is_float, double* out, cudaStream_t s);
int launch_from_double(long long n, const double* in, void* out, int out_is_float, cudaStream_t s);
int launch_split(long long n, const double* in, float* hi, float* lo, cudaStream_t s);
int launch_zero_dirichlet(const GridDev& g, double* u64, float* uhi, float* ulo, cudaStream_t s);
int launch_join(long long n, const float* hi, const float* lo, double* out, cudaStream_t s);
int min_jacobian_blocks(const GridDev& g);
int launch_min_jacobian(const GridDev& g, const double* u, const double eps[3][3], double* block_min,
                        cudaStream_t s);
int launch_stress_out(const GridDev& g, const double* u, const uint8_t* phase, const double* lam,
                      const double* mu, const double eps[3][3], int full, double* out, cudaStream_t s);

}  // namespace dtt

// Host-side state of one cell (dtt_grid of include/dtt.h), shared by the source files of
// the library that need a grid's buffers (the solver API and the warm-start network).
#pragma once
#include <string>
#include <vector>

#include "dtt.h"
#include "dtt_internal.cuh"

using dtt::Ctrl;
using dtt::FftAxisInfo;
using dtt::GridDev;
using dtt::TzComp;

struct dtt_grid {
  GridDev g{};
  int prec = DTT_PREC_FP64;
  cudaStream_t stream = nullptr;
  int device = -1;           // the device that was current at dtt_grid_create
  bool own_stream = false;   // created here when the caller passes NULL (graph capture
                             // needs a stream other than the legacy default stream)
  int types[3][3]{};      // [comp][axis]
  bool has_null[3]{};
  long long NN = 0, NV = 0;
  size_t esz = 8;

  // nodal fields
  double* u64 = nullptr;
  float* uhi = nullptr;
  float* ulo = nullptr;
  // Anderson rings (T fields): A = p ring (ACV on p~, slots 0..3) or u~-copy ring (ACV on
  // u~, slots 0..4); Gr = Green-input ring (ACV on p~) whose slot 0 is the Green input
  // otherwise; R = Anderson residual ring.  step = last full step of u~.
  void* S[5]{};
  void* R[4]{};
  void* Gr[4]{};
  void* step = nullptr;
  void* gbuf = nullptr;    // = Gr[0]
  void* spec = nullptr;
  void* spec2 = nullptr;
  void** d_Sring = nullptr;
  void** d_Rring = nullptr;
  void** d_Gring = nullptr;
  void** d_Gown = nullptr;    // the own Green-input buffers (d_Gring entries may alias the p ring)

  // material
  uint8_t* phase = nullptr;
  double* d_lam = nullptr;
  double* d_mu = nullptr;
  int nphase = 0;
  bool mat_set = false;
  double lam0 = 0, mu0 = 0;
  bool ref_set = false;
  double eps[3][3]{};

  // transforms
  FftAxisInfo fft[3]{};
  void* fft_tw[3]{};
  void* fft_ph[3]{};
  void* fft_tw1[3]{};          // stage-1 twiddles of the warp-register passes
  void* fwd[3][3]{};
  void* inv[3][3]{};
  double* sin2q[3][3]{};
  double* cos2q[3][3]{};
  float* sin2q_f[3][3]{};   // FP32 copies (mixed-precision Green multiply)
  float* cos2q_f[3][3]{};
  // tensor-core z pass (mixed path): per component the packed forward and inverse
  // matrices (one allocation, forward first), their ranges, and the route choice
  float* tz_mat[3]{};
  TzComp tz[3]{};
  bool tz_ok = false;          // every component's z operand fits (size <= 256)
  int z_route = 0;             // 0: FFT (or dense) z pass, 1: tensor-core contractions
  int fft_warp = 1;            // 1: warp-register Green step where the grid allows it
  int exact_ok = 1;            // 0 (DTT_EXACT_R=0): keep R = p - g + A0 Delta in the mixed path
  int2* d_tile_z = nullptr;    // per xy tile of the mixed residual kernel: z range of marked nodes
  int tile_cap = 0;
  int res_split = 0;           // ResidualArgs::split of the exact mode, from the marked z ranges
  unsigned int* tz_err = nullptr;
  // isotropic reference medium (Section 3.2.3): per-axis tables of sin^2(q/2), cos^2(q/2)
  // shared by the components, and per position the components with a mode there (bit c)
  double* iso_s[3]{};
  double* iso_c[3]{};
  float* iso_sf[3]{};
  float* iso_cf[3]{};
  uint8_t* iso_valid[3]{};

  // constraints (host copy + device CSR)
  int nrows = 0;
  std::vector<int> h_ptr;
  std::vector<long long> h_dof;
  std::vector<double> h_a, h_b, h_val, h_ab, h_aa;
  int* d_ptr = nullptr;
  long long* d_dof = nullptr;
  double *d_a = nullptr, *d_b = nullptr, *d_target = nullptr, *d_mult = nullptr, *d_ab = nullptr,
         *d_aa = nullptr;
  uint8_t* cmask = nullptr;

  // contact
  bool contact = false;
  int c_axis = 2, c_face = 1;
  double center[3]{}, radius = 0;
  int nface = 0;
  bool contact_given = false;   // the next start keeps the zone set by dtt_set_initial_contact
  bool fallback_saved = false;  // a guess was set over u~ of the previous increment, kept in
                                // the R ring as the fallback start of DTT_INIT_GUESS
  uint8_t* d_active_saved = nullptr;
  long long* d_face = nullptr;
  uint8_t *d_active = nullptr, *d_vgap = nullptr, *d_vreact = nullptr, *d_vgap_prev = nullptr,
          *d_vreact_prev = nullptr;
  double *d_gap = nullptr, *d_fn = nullptr, *d_nvec = nullptr;

  // control
  Ctrl* d_ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;   // pinned
  double* d_part = nullptr;
  size_t part_cap = 0;

  // scratch for operator entry points
  double* op_d = nullptr;   // 3 NN doubles
  void* op_t1 = nullptr;    // 3 NN of T
  void* op_t2 = nullptr;

  // graph
  cudaGraphExec_t gexec = nullptr;
  int g_key = -1;
  bool g_loop = false;         // gexec runs the whole solve (conditional WHILE node around the iterations)
  int* d_rounds = nullptr;     // rounds of the device-side loop (reset before each launch)
  unsigned long long id = 0;        // unique per grid of the process
  unsigned long long version = 0;   // bumped whenever captured launch arguments go stale

  Ctrl last{};
  int start_guess = 0;      // last solve started from the supplied guess (DTT_INIT_GUESS)
  double start_r = 0.0;     // Eq. 5 residual of that solve's starting iterate
  bool solved = false;
};

namespace dtt {
// sets the thread's last-error message and returns s (dtt_last_error reads it)
dtt_status set_error(dtt_status s, const std::string& msg);
}  // namespace dtt

namespace dtt {
// Writes a guess of u~ (device, 3 x n_nodes float64) over the current u~, keeping the
// current u~ as the fallback start of the next DTT_INIT_GUESS solve; with `active`
// (device, n_surface bytes) the guess's initial contact zone as well.
dtt_status set_guess_with_fallback(dtt_grid* G, const double* u_dev, const uint8_t* active_dev);
}  // namespace dtt

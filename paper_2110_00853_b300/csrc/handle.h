// Private to the library: the handle behind the cmles_handle of the C ABI,
// and the host helpers shared by api.cu (single-domain handles) and group.cu
// (a mesh split into (x, y) partitions with halo exchange).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "cmles.h"
#include "common.cuh"
#include "launch.h"
#include "mlp.cuh"

using namespace cmles;

// Chunks of an asynchronous host download (about 380 MB each for the 12 GB
// state of the 256M-node box: an upload that follows it lags by one chunk).
constexpr int kFetchChunks = 32;

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

struct cmles_t {
  cmles_mesh mesh;
  cmles_params prm;
  int N = 4, Nq = 5, Np = 125;
  // E interior elements (nodes = E Np); on a partition of a cmles_group the
  // buffers hold Es >= E storage elements (snodes = Es Np), the interior plus
  // one ghost element on each side in x and y; otherwise Es = E
  long long E = 0, nodes = 0, Es = 0, snodes = 0;
  bool part = false;
  cudaStream_t stream = 0;
  std::string err;
  std::vector<double> xi, w, D;
  KParams K;
  double *Q[2] = {nullptr, nullptr};
  int cur = 0;
  double *dQ = nullptr, *F2 = nullptr;
  double *TH64[2] = {nullptr, nullptr};  // FP64 path: thermodynamic fields of Q[i]
  // FP32 path: shadow ping-pong, FP32 LSRK register, FP32 F2/aux, tables
  bool fp32 = false;
  float *S32[2] = {nullptr, nullptr};
  float *TH32[2] = {nullptr, nullptr};  // thermodynamic fields of S32[i]
  int scur = 0;
  bool shadow_valid = false;  // FP32: S32[scur] and TH32[scur] are Q's; FP64: TH64[cur] is Q[cur]'s
  float *dQ32 = nullptr, *D32 = nullptr, *F2_32 = nullptr, *lev32 = nullptr, *dH32 = nullptr;
  double *qref64 = nullptr;
  double *rho_r = nullptr, *p_r = nullptr, *qt_r = nullptr, *tau_lev = nullptr, *tau_col = nullptr;
  double *wq = nullptr, *partials = nullptr, *budget_out = nullptr, *prof = nullptr;
  int *flags = nullptr;
  int budget_nblocks = 1;
  bool have_ref = false;
  long long launches = 0, steps = 0;
  int tc_stall = 0;
  // HEVI: level reference (host copy), stage buffers R0 R1 R2 L0 L1 B Y and
  // the tables of the vertical operator for the step hv_dt
  std::vector<double> ref_rho_h, ref_p_h, ref_qt_h;
  double *hv_buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double *hv_tab = nullptr;
  double hv_dt = -1.0;
  HeviTables hv_T{};
  // double-buffered host uploads: staging buffer, copy stream and events
  double *Qstage = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t staged_ev = nullptr, compute_ev = nullptr;
  bool staged = false;
  // asynchronous host downloads (cmles_fetch_state_host): chunked copies on
  // their own stream with one event per chunk, so that an upload of the same
  // host buffer can follow chunk by chunk
  cudaStream_t d2h_stream = nullptr;
  cudaEvent_t fetch_ev[kFetchChunks] = {};
  cudaEvent_t fetch_start_ev = nullptr, fetch_done_ev = nullptr;
  const double *fetch_src = nullptr;  // device buffer read by the latest download
  const double *fetch_host = nullptr; // host buffer it writes
  bool fetch_pending = false;         // issued and not yet waited for (cmles_wait_fetch)
  bool fetch_unordered = false;       // the handle's stream is not yet ordered after it
  double time = 0.0;
  bool timing = false;
  std::vector<TimedLaunch> timed;
  long long tcount[3] = {0, 0, 0};
  double tms[3] = {0, 0, 0};
  long long bytes = 0;
  std::vector<float> mlp;
  MlpPacked *mlp_dev = nullptr;
  ExpFilter expf = {};
  double *rvs_tab = nullptr;
  double *exr = nullptr;  // (p_r/p0)^-kappa per node level
  bool have_mlp = false;
  // curvilinear (warped) meshes: device tables and host geometry (FP64)
  bool curved = false;
  float *geo32 = nullptr, *node32 = nullptr;
  double *wJn = nullptr;
  std::vector<double> hx_, hz_, hJ_, hJa_, hdelta_;
  std::vector<double> hvr_;  // warped meshes: Vreman's Delta_m^2 per element (x, y, z)
};

namespace cmles_host {

cmles_status fail(cmles_handle h, cmles_status st, const std::string &msg);
cmles_status dalloc(cmles_handle h, void **p, size_t bytes);

// launch bookkeeping: count every kernel; with timing on, bracket by events
struct LaunchScope {
  cmles_handle h;
  int kind, nk;
  TimedLaunch tl;
  LaunchScope(cmles_handle h_, int kind_, int nkernels);
  ~LaunchScope();
};

// One partition of a larger mesh: the global mesh, the global indices of the
// first interior element and the sides (0 -x, 1 +x, 2 -y, 3 +y) that are
// walls of the global mesh.
struct PartSpec {
  cmles_mesh global;
  int gx0, gy0;
  int wall[4];
};

// cmles_create for a whole mesh (ps null) or for one partition (mesh = the
// partition's interior elements as a mesh of their own extent and origin).
cmles_status create_handle(const cmles_mesh *mesh, const cmles_params *params, const PartSpec *ps,
                           cmles_handle *out);
// FP32: the shadow of the FP64 state Q (and its thermodynamic fields) into
// buffer i; FP64: the thermodynamic fields of Q into TH.
cmles_status write_shadow(cmles_handle h, const double *Q, int i);
cmles_status write_thermo64(cmles_handle h, const double *Q, double *TH);
// the shadow or thermodynamic fields of the handle's state, when it changed
cmles_status ensure_shadow(cmles_handle h);
// the 2N-storage tables of the handle's explicit integrator
int lsrk_tables(cmles_handle h, const double **A, const double **B);

}  // namespace cmles_host

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(h, CMLES_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

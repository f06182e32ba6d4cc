// rb_api_internal.h -- host-side structures shared by the C ABI translation
// units (rb_api.cu, rb_server.cpp).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "rb.h"
#include "rb_internal.cuh"

namespace rb {

// NVTX range over one ABI call: named ranges in profiler timelines (nsys,
// ncu's --nvtx filters); without a tool attached a push/pop costs a few
// nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define RB_NVTX(name) ::rb::NvtxRange rb_nvtx_range_(name)

// Host record of one event and the device memory it owns.
struct EventEntry {
  int n_det = 0, n_bins = 0;
  int64_t kmin = 0, N = 0;
  double T = 0, f_low = 0, f_high = 0, gmst = 0;
  int bin_scheme = RB_BINS_PN;
  double epsilon = 0;  // the placement measure's range over the band / n_bins
  double theta_ref[kNPar] = {};
  double geom[kMaxDet][5] = {};  // site rows as given: lat, lon, elevation, x/y arm azimuths
  EventConst ec{};
  EventDev dev{};
  int64_t* d_edges = nullptr;
  double* d_summ = nullptr;
  float* d_tab32 = nullptr;
  float* d_slot32 = nullptr;  // slot image of the float-float mixed kernel
  double* d_tab64 = nullptr;
  RefValues* d_ref = nullptr;
  double* d_base = nullptr;
  double* d_data = nullptr;   // resident strain [D][N][2]
  double* d_psd = nullptr;    // resident PSD [D][N]
  double* d_h0 = nullptr;     // stored fiducial waveform h0_d(f) [D][N][2] (FP64 builds)
  bool h0_valid = false;      // d_h0 holds h0 for the current theta_ref
  double* d_theta_ref = nullptr;
  void* d_chunkq = nullptr;   // event-constant per-chunk Taylor matrices (fast summary build)
  void* d_chunks = nullptr;   // per-rebuild chunk records (rebuild + batch step)
  double* d_invdf = nullptr;  // [B] 1 / bin width
  double* d_share = nullptr;  // [D][B] per-bin shares of log L(theta_ref)
  SummarySync* d_sync = nullptr;  // build counters (zero between builds)
  void* d_w32 = nullptr;          // fast build: FP32 copy w = d'/S' [D][N] (float2)
  float* d_is32 = nullptr;        // fast build: FP32 copy 1/S' [D][N]
  int* d_wexp = nullptr;          // fast build: power-of-two scales {sd, sS} per detector
  bool w32_resident = false;      // the FP32 copy holds the resident data
  bool w32_current = false;       // the FP32 copy holds the data the last rebuild summed
  bool last_in_place = false;     // the last rebuild read caller data in place
  cudaStream_t side = nullptr;    // rebuild: branch for the reference values the summary does not use
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_ref = nullptr;   // rebuild + batch: float-float reference values ready
  cudaEvent_t ev_setup = nullptr; // rebuild + batch: the walkers' set-up done (forked stream)
  // rebuild + batch: the walkers' workspace, kept between calls (grown outside
  // stream capture only; outgrown buffers stay allocated until the event is
  // freed, so a captured graph never refers to freed memory)
  void* step_ws = nullptr;
  size_t step_ws_bytes = 0;
  void* step_ws_old[16] = {};
  int n_step_ws_old = 0;
  cudaStream_t tanst = nullptr;   // rebuild + batch: the walkers' tangents
  cudaEvent_t ev_tan = nullptr;
  cudaStream_t copy = nullptr;    // host-buffer rebuild + batch: strain/PSD copies in
  cudaEvent_t ev_data = nullptr;  // ... and their completion
  // host-buffer batch with pinned walkers and outputs: its set-up and
  // likelihood launches, captured once for (buffers, W, mode) and replayed
  cudaGraphExec_t hg_exec = nullptr;
  cudaStream_t hg_stream = nullptr;  // the capture stream
  const double* hg_theta = nullptr;
  double* hg_logl = nullptr;
  double* hg_grad = nullptr;
  int64_t hg_W = 0;
  int hg_mode = -1;
  void* hg_ws = nullptr;             // the captured launches' workspace
  size_t hg_ws_bytes = 0;
  // host-buffer rebuild + batch with everything pinned: the whole call
  // (host-link read, rebuild, batch), captured once per buffers and replayed
  cudaGraphExec_t hs_exec = nullptr;
  const double* hs_data[RB_MAX_DET] = {};
  const double* hs_psd[RB_MAX_DET] = {};
  const double* hs_theta = nullptr;
  double* hs_logl = nullptr;
  double* hs_grad = nullptr;
  int64_t hs_W = 0;
  int hs_mode = -1;
  uint64_t hs_launches = 0;
  PartDesc* d_parts = nullptr;    // fast build: parts of bins
  float* d_part_sums = nullptr;   // fast build: per-part float-pair sums
  int n_parts = 0;
  size_t device_bytes = 0;
  uint64_t uid = 0;  // unique per built event (never reused within a process)
  SummaryOut out() const {
    return SummaryOut{d_summ, d_tab32 + dev.edge32_floats, d_tab64 + (size_t)(kNBasis + 1) * dev.e_pad, d_invdf,
                      d_share, d_sync, d_base, dev.b_pad, d_parts, d_part_sums, n_parts,
                      d_slot32 + (size_t)4 * (kNBasis + 1) * dev.n_slots, dev.n_slots};
  }
};

const EventEntry* event_entry(::rb_event_s* ev);

int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void count_launches(uint64_t n);
int sm_count();

// Per-walker workspace of one batch, in bytes per walker.
size_t walker_ws_bytes(int mode, bool grad);

// Set-up + likelihood kernels for one batch; scratch = NULL takes the
// workspace from the stream-ordered allocator.  With mala, the likelihood
// kernel finishes each walker with the MALA accept step (logl, grad unused).
int run_batch(const EventEntry* e, const double* theta, int64_t W, double* logl, double* grad, int mode,
              cudaStream_t s, void* scratch, const MalaArgs* mala = nullptr);

// Fiducial values, summary data, tables and base of an event from the given
// device strain/PSD (NULL: the event's resident copy); no allocation, no
// synchronisation.
// mode RB_FP64 uses the FP64 summary kernel; the mixed modes use the fast
// Taylor-chunk kernel when T f_low >= 1024 and N <= 2^30 (FP64 kernel otherwise).
// The walkers' set-up of a batch that follows a rebuild on the same stream
// (rb_rebuild_loglike_grad): it needs only the reference values and theta, so
// the rebuild runs it on its forked stream, overlapped with the summary sums.
struct SideSetup {
  const double* theta;
  int64_t W;
  void* ws;
  void* tan;
  bool grad;
  cudaEvent_t data_ready;  // if not NULL: the resident data are complete only after this event
};
int rebuild_event(EventEntry& e, const DataPtrs* in, int mode, cudaStream_t s, const SideSetup* side_setup = nullptr);
// Stream-ordered allocation from the library's memory pool (see rb_api.cu).
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s);
int rebuild_and_batch(EventEntry& e, const double* theta, int64_t W, double* logl, double* grad, int mode,
                      cudaStream_t s, cudaEvent_t data_ready);
// The likelihood kernel of a batch whose set-up has been done (trace events around it).
cudaError_t launch_batch_main(const EventEntry* e, void* ws, void* tan, int64_t W, double* logl, double* grad, int mode,
                              cudaStream_t s, const MalaArgs* mala);

// Events recorded on the launch stream right before / after the main
// likelihood kernel of every batch (NULL disables).
void set_trace_events(void* before, void* after);

}  // namespace rb

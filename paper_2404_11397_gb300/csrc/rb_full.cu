// rb_full.cu -- the full (unbinned) log-likelihood of Eqs. 2-3 for a batch
// of walkers, on the full frequency grid: the quantity relative binning
// approximates, used for the reference-parameter search and for checking the
// binned likelihood (Sec. II.C; Sec. III.A).
//
// With the Newtonian amplitude the waveform is h_d(f; theta) = K_d(theta)
// f^-7/6 exp(-2 pi i x_d(f; theta)), so per detector
//   <d|h> = 4 df Re[conj(K_d) Z_d],  Z_d = sum_k (d_k / S_k) f_k^-7/6 exp(+2 pi i x_d(f_k)),
//   <h|h> = |K_d|^2 H_d,             H_d = 4 df sum_k f_k^-7/3 / S_k,
//   log L = sum_d (<d|h> - <h|h> / 2).
// H_d does not depend on theta: it is sum_b B0_{d,b} / |K_d(theta_ref)|^2 from
// the summary data (B0 = <h0|h0> over the bin).  Z_d is the expensive part: a
// walker-dependent phase at every grid point.  It is evaluated like the fast
// summary build: x_d on a chunk of 32 points is a Taylor polynomial whose
// coefficients are the walker's c_k / 2pi contracted with the event's chunk
// matrices, and the delay enters as exp(2 pi i f_c tau_d) exp(2 pi i j df tau_d).
//
// Mapping: a block of 8 warps owns 8 walkers (one per warp) and one slice of
// the grid (blockIdx.y), which it walks in segments of 32 chunks (1024
// points); the number of slices is picked so the grid fills whole waves.  Per
// segment the block stages the chunk matrices and the FP32 data copy times
// f^-7/6 in shared memory, the data transposed (read once for the 8 walkers;
// the event's data stay in L2).  Lane c of a warp forms its walker's Taylor
// coefficients and chunk factors exp(2 pi i f_c tau_d) for chunk c, keeps them
// in registers and walks the chunk's 32 points; the offset factors
// exp(2 pi i (j - 16) df tau_d), the same for all lanes at a given offset j,
// come from a per-warp table (broadcast loads), and the chunk factor is
// applied once to the chunk's sum.  Per point: the phase polynomial, one
// sin/cos, and per detector the offset factor times the phasor times the
// data.  Per-lane sums are FP32 per chunk, accumulated in float pairs; the
// warp sum and the final combination are FP64.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "rb.h"
#include "rb_api_internal.h"
#include "rb_internal.cuh"

namespace rb {

constexpr int kFullWarps = 8;
constexpr int kFullThreads = kFullWarps * 32;
constexpr int kSegC = 32;                 // chunks per segment
constexpr int kSegP = kSegC * kChunk;     // points per segment
constexpr int kWtRow = kSegC + 1;       // transposed data row (padded: conflict-free stores)
constexpr int kQPad = kQRow + 1;        // staged chunk-matrix row (padded: lane c reads row c without conflicts)
constexpr size_t kFullSmem = sizeof(float) * (kSegC * kQPad + 4) + (sizeof(float4) + sizeof(float2)) * kChunk * kWtRow +
                             (sizeof(float4) + sizeof(float2)) * kFullWarps * kChunk;

// Per slice and walker: the slice's part of Z_d (complex, 3 detectors) as
// FP64 in zout[slice][w][6].  ND = number of detectors.
template <int ND>
__global__ void __launch_bounds__(kFullThreads) k_full_z(const float2* __restrict__ w32, int N,
                                                        const float* __restrict__ q, int n_chunks,
                                                        const WalkerAbs* __restrict__ wabs, int64_t W,
                                                        float invT_hi, float invT_lo, int seg_per_slice,
                                                        double* __restrict__ zout) {
  // dynamic shared memory: the segment's chunk matrices; its data times
  // f^-7/6 transposed, for point c * 32 + j of the segment at [j][c] --
  // detectors 0 and 1 as {re_0, re_1, im_0, im_1} (wp), the single detector
  // D-1 as {re, im} (ws); and per warp the walker's offset factors
  // exp(2 pi i (j - 16) df tau_d) in the same two forms (tp, ts)
  extern __shared__ __align__(16) unsigned char smem_full[];
  float* qs = reinterpret_cast<float*>(smem_full);
  float4 (*wp)[kWtRow] = reinterpret_cast<float4 (*)[kWtRow]>(qs + kSegC * kQPad + 4 - (kSegC * kQPad) % 4);
  float2 (*ws)[kWtRow] = reinterpret_cast<float2 (*)[kWtRow]>(wp + kChunk);
  float4 (*tp)[kChunk] = reinterpret_cast<float4 (*)[kChunk]>(ws + kChunk);
  float2 (*ts)[kChunk] = reinterpret_cast<float2 (*)[kChunk]>(tp + kFullWarps);
  constexpr bool kPair = ND >= 2;
  constexpr int kSingle = (ND & 1) ? ND - 1 : -1;
  constexpr int D = ND;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t w = (int64_t)blockIdx.x * kFullWarps + warp;
  const bool live = w < W;
  // the walker's absolute values (float pairs)
  float ch[kNBasis][2], p0[2], tt[kMaxDet][2];
  int valid = 0;
  if (live) {
    const WalkerAbs& a = wabs[w];
    for (int k = 0; k < kNBasis; ++k) { ch[k][0] = a.chat[k][0]; ch[k][1] = a.chat[k][1]; }
    p0[0] = a.phi0t[0];
    p0[1] = a.phi0t[1];
    for (int d = 0; d < kMaxDet; ++d) { tt[d][0] = a.taut[d][0]; tt[d][1] = a.taut[d][1]; }
    valid = a.valid;
  } else {
    for (int k = 0; k < kNBasis; ++k) ch[k][0] = ch[k][1] = 0.f;
    p0[0] = p0[1] = 0.f;
    for (int d = 0; d < kMaxDet; ++d) tt[d][0] = tt[d][1] = 0.f;
  }
  // offset factors of the walker: lane j forms exp(2 pi i (j - 16) df tau_d)
  {
    const float jf = small_int_float(lane - kChunk / 2);
    float2 t[kMaxDet];
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      float sh = 0.f, sl = 0.f;
      f2x_fma_acc(tt[d][0], tt[d][1], invT_hi, invT_lo, sh, sl);  // tau_d df
      const float p = __fmul_rn(sh, jf);
      const float e = __fmaf_rn(sl, jf, __fmaf_rn(sh, jf, -p));
      t[d] = cis_turns(frac_turns(p, e));
    }
    tp[warp][lane] = make_float4(t[0].x, t[1].x, t[0].y, t[1].y);
    ts[warp][lane] = t[kSingle < 0 ? 0 : kSingle];
  }
  float zh[kMaxDet][2], zl[kMaxDet][2];  // Z_d as float pairs (re, im)
  for (int d = 0; d < kMaxDet; ++d) zh[d][0] = zh[d][1] = zl[d][0] = zl[d][1] = 0.f;
  const int n_seg = (n_chunks + kSegC - 1) / kSegC;
  const int sg0 = blockIdx.y * seg_per_slice, sg1 = min(n_seg, sg0 + seg_per_slice);
  for (int sg = sg0; sg < sg1; ++sg) {
    const int c0 = sg * kSegC, nc = min(kSegC, n_chunks - c0);
    __syncthreads();  // the previous segment is no longer read (and tw is written)
    {
      const float* src = q + (size_t)c0 * kQRow;
      for (int i = tid; i < nc * kQRow; i += kFullThreads) {
        const int c = i / kQRow;
        qs[c * kQPad + (i - c * kQRow)] = __ldg(src + i);
      }
    }
    __syncthreads();
    // data times f^-7/6 = f_c^-7/6 (1 + j u)^-7/6 (chunk series), transposed;
    // points past the grid are zero
    for (int p = tid; p < kSegP; p += kFullThreads) {
      const int c = p >> 5, jj = p & (kChunk - 1);
      const int k = c0 * kChunk + p;
      float2 v[kMaxDet] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (c < nc && k < N) {
        const float* qa = qs + c * kQPad + kQamp;
        const float j = small_int_float(jj - kChunk / 2);
        const float A = qa[0] * fmaf(j, fmaf(j, fmaf(j, fmaf(j, qa[4], qa[3]), qa[2]), qa[1]), 1.f);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float2 x = __ldg(w32 + (size_t)d * N + k);
          v[d] = make_float2(x.x * A, x.y * A);
        }
      }
      if (kPair) wp[jj][c] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
      if (kSingle >= 0) ws[jj][c] = v[kSingle < 0 ? 0 : kSingle];
    }
    // lane c: the walker's coefficients of chunk c (X0 with Phi0, whole turns
    // dropped) and the chunk factors exp(2 pi i f_c tau_d), in registers
    float X0h = 0.f, X0l = 0.f, X1h = 0.f, X1l = 0.f, X2h = 0.f, X2l = 0.f, xn[kOrd - 2];
    float2 E[kMaxDet];
#pragma unroll
    for (int n = 0; n < kOrd - 2; ++n) xn[n] = 0.f;
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) E[d] = make_float2(1.f, 0.f);
    const bool act = live && valid && lane < nc;
    if (act) {
      const float* row = qs + lane * kQPad;
      X0h = p0[0];
      X0l = p0[1];
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) {
        const float a = ch[k][0], b = ch[k][1];
        f2x_fma_acc(a, b, row[kQ01 + 4 * k], row[kQ01 + 4 * k + 1], X0h, X0l);
        f2x_fma_acc(a, b, row[kQ01 + 4 * k + 2], row[kQ01 + 4 * k + 3], X1h, X1l);
        f2x_fma_acc(a, b, row[kQ2 + 2 * k], row[kQ2 + 2 * k + 1], X2h, X2l);
#pragma unroll
        for (int n = 0; n < kOrd - 2; ++n) xn[n] = fmaf(a, row[kQh + n * kNBasis + k], xn[n]);
      }
      X0h = __fadd_rn(X0h, -round_fma_pipe(X0h));
      const float fch = row[kQfc], fcl = row[kQfc + 1];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        float ah = 0.f, al = 0.f;
        f2x_fma_acc(tt[d][0], tt[d][1], fch, fcl, ah, al);  // f_c tau_d
        E[d] = cis_turns(frac_turns(ah, al));
      }
    }
    __syncthreads();  // wt complete
    if (!act) continue;
    float2 apr = make_float2(0.f, 0.f), api = apr;  // detectors 0, 1
    float asr = 0.f, asi = 0.f;                     // detector D-1
#pragma unroll 2
    for (int jj = 0; jj < kChunk; ++jj) {
      const float jf = small_int_float(jj - kChunk / 2);
      // x = X0 + X1 j + X2 j^2 + j^3 (X3 + ... + X8 j^5)
      const float t = fmaf(fmaf(fmaf(fmaf(fmaf(xn[5], jf, xn[4]), jf, xn[3]), jf, xn[2]), jf, xn[1]), jf, xn[0]);
      const float j2 = jf * jf;
      const float t3 = t * (j2 * jf);
      const float p1 = __fmul_rn(X1h, jf);
      float e1 = __fmaf_rn(X1h, jf, -p1);
      e1 = __fmaf_rn(X1l, jf, e1);
      const float p2 = __fmul_rn(X2h, j2);
      float e2 = __fmaf_rn(X2h, j2, -p2);
      e2 = __fmaf_rn(X2l, j2, e2);
      float sh = X0h, sl = X0l;
      f2x_add(sh, sl, p1);
      f2x_add(sh, sl, p2);
      sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e1, e2), t3));
      const float2 z = cis_turns(frac_turns(sh, sl));  // exp(+2 pi i x)
      // offset factor exp(2 pi i (j - 16) df tau_d) (the same for all lanes)
      // times the phasor, times the data
      if constexpr (kPair) {
        const float4 T = tp[warp][jj];
        const float4 v = wp[jj][lane];
        const float2 Tr = make_float2(T.x, T.y), Ti = make_float2(T.z, T.w);
        const float2 zx = make_float2(z.x, z.x), zy = make_float2(z.y, z.y);
        const float2 ur = pv::fma(zx, Tr, pv::mul(pv::neg(zy), Ti)), ui = pv::fma(zx, Ti, pv::mul(zy, Tr));
        const float2 vr = make_float2(v.x, v.y), vi = make_float2(v.z, v.w);
        apr = pv::fma(vr, ur, pv::fma(pv::neg(vi), ui, apr));
        api = pv::fma(vr, ui, pv::fma(vi, ur, api));
      }
      if constexpr (kSingle >= 0) {
        const float2 T = ts[warp][jj];
        const float ur = fmaf(z.x, T.x, -z.y * T.y), ui = fmaf(z.x, T.y, z.y * T.x);
        const float2 v = ws[jj][lane];
        asr = fmaf(v.x, ur, fmaf(-v.y, ui, asr));
        asi = fmaf(v.x, ui, fmaf(v.y, ur, asi));
      }
    }
    // the chunk factor, once per chunk, then into the lane's float pairs
    float acc[kMaxDet][2] = {{apr.x, api.x}, {apr.y, api.y}, {0.f, 0.f}};
    if (kSingle >= 0) {
      acc[kSingle < 0 ? 0 : kSingle][0] = asr;
      acc[kSingle < 0 ? 0 : kSingle][1] = asi;
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float gr = fmaf(E[d].x, acc[d][0], -E[d].y * acc[d][1]);
      const float gi = fmaf(E[d].x, acc[d][1], E[d].y * acc[d][0]);
      f2x_add(zh[d][0], zl[d][0], gr);
      f2x_add(zh[d][1], zl[d][1], gi);
    }
  }
  if (!live) return;
  double* zo = zout + ((size_t)blockIdx.y * W + w) * 6;
  // warp sums in FP64 (lane order fixed by the butterfly)
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    const double re = warp_sum_f64((double)zh[d][0] + (double)zl[d][0]);
    const double im = warp_sum_f64((double)zh[d][1] + (double)zl[d][1]);
    if (lane == 0) {
      zo[2 * d] = valid ? re : 0.0;
      zo[2 * d + 1] = valid ? im : 0.0;
    }
  }
  if (lane == 0 && !valid) zo[0] = NAN;  // marks an unphysical walker
}

// log L per walker from Z_d and K_d (FP64); H_d from the summary's B0 and
// the reference prefactor, scales from the FP32 data copy's exponents.
__global__ void __launch_bounds__(128) k_full_finish(const double* __restrict__ zout, int n_slices,
                                                     const WalkerAbs* __restrict__ wabs,
                                                     int64_t W, int D, int B, double T, const int* __restrict__ exps,
                                                     const double* __restrict__ summ, const RefValues* __restrict__ ref,
                                                     double* __restrict__ logl) {
  __shared__ double H[kMaxDet], sc0[kMaxDet];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int d = 0; d < D; ++d) {
      double s = 0.0;
      for (int b = lane; b < B; b += 32) s += summ[((size_t)d * B + b) * 6 + 4];  // B0
      s = warp_sum_f64(s);
      if (lane == 0) {
        const double kr = ref->K[d][0], ki = ref->K[d][1];
        H[d] = s / (kr * kr + ki * ki);
        const int sd = exps[2 * d], sS = exps[2 * d + 1];
        sc0[d] = (4.0 / T) * __hiloint2double((1023 + sS - sd) << 20, 0);
      }
    }
  }
  __syncthreads();
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  if (!wabs[w].valid) {
    logl[w] = -INFINITY;
    return;
  }
  double z[2 * kMaxDet] = {0, 0, 0, 0, 0, 0};
  for (int sl = 0; sl < n_slices; ++sl) {  // slices in order: the sum does not depend on the schedule
    const double* zs = zout + ((size_t)sl * W + w) * 6;
#pragma unroll
    for (int i = 0; i < 2 * kMaxDet; ++i)
      if (i < 2 * D) z[i] += zs[i];
  }
  double L = 0.0;
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    if (d >= D) break;
    const double kr = wabs[w].K[d][0], ki = wabs[w].K[d][1];
    const double dh = sc0[d] * (kr * z[2 * d] + ki * z[2 * d + 1]);  // Re(conj(K) Z)
    L += dh - 0.5 * (kr * kr + ki * ki) * H[d];
  }
  logl[w] = L;
}

cudaError_t launch_setup_abs(const double* theta, int64_t W, const EventConst& ec, WalkerAbs* out, cudaStream_t s);
cudaError_t launch_data32(const DataPtrs& in, int64_t N, int D, void* w32, float* is32, int* exps, cudaStream_t s);

}  // namespace rb

extern "C" int rb_loglike_full_batch(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev, int mode,
                                     void* stream) {
  RB_NVTX("rb_loglike_full_batch");
  using namespace rb;
  if (!ev) return set_error(RB_EINVAL, "rb_loglike_full_batch: NULL event");
  if (W < 0) return set_error(RB_EINVAL, "rb_loglike_full_batch: W < 0");
  if (W == 0) return RB_OK;
  if (!theta_dev || !logl_dev) return set_error(RB_EINVAL, "rb_loglike_full_batch: NULL theta or logl");
  if (mode != RB_MIXED) return set_error(RB_EINVAL, "rb_loglike_full_batch: only RB_MIXED is provided");
  EventEntry& e = *const_cast<EventEntry*>(event_entry(ev));
  if (!(e.kmin >= 1024 && e.N <= (int64_t(1) << 30)))
    return set_error(RB_EINVAL, "rb_loglike_full_batch: needs T f_low >= 1024 and N <= 2^30 (chunk expansion)");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err;
  if (!e.w32_current) {  // FP32 working copy of the data the summary was built from
    if (e.last_in_place)
      return set_error(RB_EINVAL,
                       "rb_loglike_full_batch: the last rebuild read caller data in place in RB_FP64 mode; "
                       "rebuild in a mixed mode or from resident data");
    DataPtrs in{};
    for (int d = 0; d < e.n_det; ++d) {
      in.data[d] = e.d_data + 2 * (size_t)d * e.N;
      in.psd[d] = e.d_psd + (size_t)d * e.N;
    }
    if ((err = launch_data32(in, e.N, e.n_det, e.d_w32, e.d_is32, e.d_wexp, s)) != cudaSuccess)
      return cuda_fail(err, "rb_loglike_full_batch: data conversion kernel");
    e.w32_resident = e.w32_current = true;
    count_launches(1);
  }
  void (*const kz)(const float2*, int, const float*, int, const WalkerAbs*, int64_t, float, float, int, double*) =
      e.n_det == 1 ? k_full_z<1> : e.n_det == 2 ? k_full_z<2> : k_full_z<3>;
  static std::atomic<bool> smem_raised[kMaxDet];  // the attribute is idempotent: concurrent first calls only repeat it
  if (!smem_raised[e.n_det - 1].load(std::memory_order_acquire)) {
    if ((err = cudaFuncSetAttribute(kz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFullSmem)) != cudaSuccess)
      return cuda_fail(err, "rb_loglike_full_batch: shared memory attribute");
    smem_raised[e.n_det - 1].store(true, std::memory_order_release);
  }
  // slices of the grid per group of 8 walkers: at least two waves of blocks
  // (2 per SM), then the count in the next few that wastes the least of the last wave
  const int nc = (int)((e.N + kChunk - 1) / kChunk);
  const int n_seg = (nc + kSegC - 1) / kSegC;
  const int64_t wblocks = (W + kFullWarps - 1) / kFullWarps;
  int n_slices = 1;
  {
    int dev = 0, n_sm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t wave = 2 * (int64_t)n_sm;
    const int64_t s_min = std::max<int64_t>(1, (2 * wave + wblocks - 1) / wblocks);
    const int64_t s_cap = std::max<int64_t>(1, n_seg / 2);  // keep >= 2 segments per slice
    double best = -1.0;
    for (int64_t sl = std::min(s_min, s_cap); sl <= std::min(s_min + 8, s_cap); ++sl) {
      const int64_t per = (n_seg + sl - 1) / sl, used = (n_seg + per - 1) / per;  // slices actually non-empty
      const int64_t blocks = wblocks * used;
      const double eff = (double)blocks / (double)(wave * ((blocks + wave - 1) / wave));
      if (eff > best + 1e-9) { best = eff; n_slices = (int)used; }
    }
  }
  const int seg_per_slice = (n_seg + n_slices - 1) / n_slices;
  char* buf = nullptr;
  const size_t abs_bytes = sizeof(WalkerAbs) * W, z_bytes = sizeof(double) * 6 * W * n_slices;
  err = ws_alloc(reinterpret_cast<void**>(&buf), abs_bytes + z_bytes, s);
  if (err != cudaSuccess) return cuda_fail(err, "rb_loglike_full_batch: workspace allocation");
  WalkerAbs* wabs = reinterpret_cast<WalkerAbs*>(buf);
  double* zout = reinterpret_cast<double*>(buf + abs_bytes);
  const double invT = 1.0 / e.T;
  const float ih = (float)invT, il = (float)(invT - (double)ih);
  int rc = RB_OK;
  if ((err = launch_setup_abs(theta_dev, W, e.ec, wabs, s)) != cudaSuccess) {
    rc = cuda_fail(err, "rb_loglike_full_batch: set-up kernel");
  } else {
    kz<<<dim3((unsigned)wblocks, (unsigned)n_slices), kFullThreads, kFullSmem, s>>>(
        static_cast<const float2*>(e.d_w32), (int)e.N, static_cast<const float*>(e.d_chunkq), nc, wabs, W, ih, il,
        seg_per_slice, zout);
    k_full_finish<<<(unsigned)((W + 127) / 128), 128, 0, s>>>(zout, n_slices, wabs, W, e.n_det, e.n_bins, e.T, e.d_wexp,
                                                              e.d_summ, e.d_ref, logl_dev);
    if ((err = cudaGetLastError()) != cudaSuccess) rc = cuda_fail(err, "rb_loglike_full_batch: kernels");
    else count_launches(3);
  }
  cudaFreeAsync(buf, s);
  return rc;
}

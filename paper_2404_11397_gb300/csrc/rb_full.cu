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
// points); the number of slices is picked so the grid fills whole waves.  Per segment the block
// stages the chunk matrices and the FP32 data copy times f^-7/6 in shared
// memory (read once for the 8 walkers; the event's data stay in L2); lane l
// of a warp forms its walker's coefficients for chunk l, then evaluates the
// points l, l + 32, ... of the segment, which all have the in-chunk offset
// j = l - 16, so its delay factor exp(2 pi i j df tau_d) is a constant that
// is applied once to the lane's sum, after the loop.  Per point: the chunk
// record (five 16-byte broadcast loads), the phase polynomial, one sin/cos,
// and per detector exp(2 pi i f_c tau_d) times the point's phasor times the
// data.  Per-lane sums are FP32 per segment, accumulated in float pairs; the
// warp sum and the final combination are FP64.
#include <algorithm>
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
constexpr int kFRec = 20;                 // floats per walker-chunk record
constexpr size_t kFullSmem = sizeof(float) * kSegC * kQRow + sizeof(float2) * kMaxDet * kSegP +
                             sizeof(float) * kFullWarps * kSegC * kFRec;

// Per slice and walker: the slice's part of Z_d (complex, 3 detectors) as
// FP64 in zout[slice][w][6].  ND = number of detectors.
template <int ND>
__global__ void __launch_bounds__(kFullThreads) k_full_z(const float2* __restrict__ w32, int N,
                                                        const float* __restrict__ q, int n_chunks,
                                                        const WalkerAbs* __restrict__ wabs, int64_t W,
                                                        float invT_hi, float invT_lo, int seg_per_slice,
                                                        double* __restrict__ zout) {
  // dynamic shared memory: chunk matrices of the segment, (d'/S') f^-7/6,
  // per-walker chunk coefficients
  extern __shared__ __align__(16) unsigned char smem_full[];
  float* qs = reinterpret_cast<float*>(smem_full);
  float2 (*wa)[kSegP] = reinterpret_cast<float2 (*)[kSegP]>(qs + kSegC * kQRow);
  float (*rec)[kSegC][kFRec] = reinterpret_cast<float (*)[kSegC][kFRec]>(wa + kMaxDet);
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
  // this lane's in-chunk offset j = lane - 16 and delay factors exp(2 pi i j df tau_d)
  const float jf = small_int_float(lane - kChunk / 2);
  float2 toff[kMaxDet];
  for (int d = 0; d < kMaxDet; ++d) {
    float sh = 0.f, sl = 0.f;
    f2x_fma_acc(tt[d][0], tt[d][1], invT_hi, invT_lo, sh, sl);  // tau_d df
    const float p = __fmul_rn(sh, jf);
    const float e = __fmaf_rn(sl, jf, __fmaf_rn(sh, jf, -p));
    toff[d] = cis_turns(frac_turns(p, e));
  }
  float zh[kMaxDet][2], zl[kMaxDet][2];  // Z_d as float pairs (re, im)
  for (int d = 0; d < kMaxDet; ++d) zh[d][0] = zh[d][1] = zl[d][0] = zl[d][1] = 0.f;
  const int n_seg = (n_chunks + kSegC - 1) / kSegC;
  const int sg0 = blockIdx.y * seg_per_slice, sg1 = min(n_seg, sg0 + seg_per_slice);
  for (int sg = sg0; sg < sg1; ++sg) {
    const int c0 = sg * kSegC, nc = min(kSegC, n_chunks - c0);
    __syncthreads();  // the previous segment is no longer read
    {
      const float4* src = reinterpret_cast<const float4*>(q + (size_t)c0 * kQRow);
      float4* dst = reinterpret_cast<float4*>(qs);
      for (int i = tid; i < nc * (kQRow / 4); i += kFullThreads) dst[i] = __ldg(src + i);
    }
    for (int i = tid; i < D * kSegP; i += kFullThreads) {
      const int d = i / kSegP, p = i - d * kSegP;
      const int k = c0 * kChunk + p;
      wa[d][p] = (k < N) ? __ldg(w32 + (size_t)d * N + k) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // amplitude f^-7/6 = f_c^-7/6 (1 + j u)^-7/6 from the chunk's series
    for (int i = tid; i < D * kSegP; i += kFullThreads) {
      const int d = i / kSegP, p = i - d * kSegP;
      const float* qa = qs + (p >> 5) * kQRow + kQamp;
      const float j = small_int_float((p & (kChunk - 1)) - kChunk / 2);
      const float A = qa[0] * fmaf(j, fmaf(j, fmaf(j, fmaf(j, qa[4], qa[3]), qa[2]), qa[1]), 1.f);
      const float2 v = wa[d][p];
      wa[d][p] = make_float2(v.x * A, v.y * A);
    }
    // this walker's coefficients of chunk `lane` (X0 with Phi0, whole turns dropped)
    if (lane < nc) {
      const float* row = qs + lane * kQRow;
      float x0h = p0[0], x0l = p0[1], x1h = 0.f, x1l = 0.f, x2h = 0.f, x2l = 0.f, xn[kOrd - 2];
#pragma unroll
      for (int n = 0; n < kOrd - 2; ++n) xn[n] = 0.f;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) {
        const float a = ch[k][0], b = ch[k][1];
        f2x_fma_acc(a, b, row[kQ01 + 4 * k], row[kQ01 + 4 * k + 1], x0h, x0l);
        f2x_fma_acc(a, b, row[kQ01 + 4 * k + 2], row[kQ01 + 4 * k + 3], x1h, x1l);
        f2x_fma_acc(a, b, row[kQ2 + 2 * k], row[kQ2 + 2 * k + 1], x2h, x2l);
#pragma unroll
        for (int n = 0; n < kOrd - 2; ++n) xn[n] = fmaf(a, row[kQh + n * kNBasis + k], xn[n]);
      }
      float* r = rec[warp][lane];
      r[0] = __fadd_rn(x0h, -round_fma_pipe(x0h));
      r[1] = x0l;
      r[2] = x1h;
      r[3] = x1l;
      r[4] = x2h;
      r[5] = x2l;
#pragma unroll
      for (int n = 0; n < kOrd - 2; ++n) r[6 + n] = xn[n];
      const float fch = row[kQfc], fcl = row[kQfc + 1];
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        float ah = 0.f, al = 0.f;
        f2x_fma_acc(tt[d][0], tt[d][1], fch, fcl, ah, al);  // f_c tau_d
        const float2 e = cis_turns(frac_turns(ah, al));
        r[12 + 2 * d] = e.x;
        r[13 + 2 * d] = e.y;
      }
    }
    __syncthreads();
    if (!live || !valid) continue;
    float acc[kMaxDet][2];
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) acc[d][0] = acc[d][1] = 0.f;
    for (int c = 0; c < nc; ++c) {
      const int p = c * kChunk + lane;
      const float4* r4 = reinterpret_cast<const float4*>(rec[warp][c]);
      const float4 qa = r4[0], qb = r4[1], qc = r4[2];  // X0 hi/lo, X1 hi/lo | X2 hi/lo, X3, X4 | X5..X8
      // x = X0 + X1 j + X2 j^2 + j^3 (X3 + ... + X8 j^5)
      const float t = fmaf(fmaf(fmaf(fmaf(fmaf(qc.w, jf, qc.z), jf, qc.y), jf, qc.x), jf, qb.w), jf, qb.z);
      const float j2 = jf * jf;
      const float t3 = t * (j2 * jf);
      const float p1 = __fmul_rn(qa.z, jf);
      float e1 = __fmaf_rn(qa.z, jf, -p1);
      e1 = __fmaf_rn(qa.w, jf, e1);
      const float p2 = __fmul_rn(qb.x, j2);
      float e2 = __fmaf_rn(qb.x, j2, -p2);
      e2 = __fmaf_rn(qb.y, j2, e2);
      float sh = qa.x, sl = qa.y;
      f2x_add(sh, sl, p1);
      f2x_add(sh, sl, p2);
      sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e1, e2), t3));
      const float2 z = cis_turns(frac_turns(sh, sl));  // exp(+2 pi i x)
      const float4 ea = r4[3];  // exp(2 pi i f_c tau_d): d = 0, 1
      const float2 eb = *reinterpret_cast<const float2*>(r4 + 4);  // d = 2
      const float er[kMaxDet] = {ea.x, ea.z, eb.x}, ei[kMaxDet] = {ea.y, ea.w, eb.y};
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float ur = fmaf(z.x, er[d], -z.y * ei[d]), ui = fmaf(z.x, ei[d], z.y * er[d]);
        const float2 v = wa[d][p];
        acc[d][0] = fmaf(v.x, ur, fmaf(-v.y, ui, acc[d][0]));
        acc[d][1] = fmaf(v.x, ui, fmaf(v.y, ur, acc[d][1]));
      }
    }
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      f2x_add(zh[d][0], zl[d][0], acc[d][0]);
      f2x_add(zh[d][1], zl[d][1], acc[d][1]);
    }
  }
  if (!live) return;
  double* zo = zout + ((size_t)blockIdx.y * W + w) * 6;
  // the lane's delay factor exp(2 pi i j df tau_d), then warp sums in FP64
  // (lane order fixed by the butterfly)
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    const double sr = (double)zh[d][0] + (double)zl[d][0], si = (double)zh[d][1] + (double)zl[d][1];
    const double tr = toff[d].x, ti = toff[d].y;
    const double re = warp_sum_f64(sr * tr - si * ti);
    const double im = warp_sum_f64(sr * ti + si * tr);
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
  static bool smem_raised[kMaxDet] = {false, false, false};  // idempotent attribute; races only repeat it
  if (!smem_raised[e.n_det - 1]) {
    if ((err = cudaFuncSetAttribute(kz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFullSmem)) != cudaSuccess)
      return cuda_fail(err, "rb_loglike_full_batch: shared memory attribute");
    smem_raised[e.n_det - 1] = true;
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

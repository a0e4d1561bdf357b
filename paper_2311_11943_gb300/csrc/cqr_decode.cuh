// cqr_decode.cuh -- a7 decode in two parts shared by the decode kernels and the batched factor
// kernel (which recovers an instance's tiles itself when the instance reaches its erasure
// panel): decode_setup builds one code's coefficient tables in shared memory (every thread of
// the CTA calls it), decode_apply recovers one position (r, s) of the code's lost tiles.
//
// Recovery Lemma (Appendix, Eq. (A_recov)), second form: each lost systematic tile is a linear
// combination of the surviving systematic tiles and the used checksum tiles, with coefficients
// from G^-1 (FP64 Gauss-Jordan with partial pivoting, one thread).  Lost checksum tiles are
// re-encoded from the systematic tiles (surviving and rebuilt).  The same code serves the
// vertical code of a Q grid column (tile index along rows) and the horizontal code of an R
// block row (along columns).  Sums run over the code tiles in ascending order.
#pragma once
#include <math.h>
#include <stdint.h>

#include "cqr_device.cuh"
#include "cqr_kernels.cuh"

namespace cqr {

template <typename T>
struct DecodeScratch {
  double Ginv[kMaxF * kMaxF];
  double a[kMaxF][2 * kMaxF];  // Gauss-Jordan tableau [G^ | I]
  T coef[kMaxF][kMaxCode];     // lost systematic b <- code tile t (nsys + f columns)
  T cenc[kMaxF][kMaxCode];     // lost checksum e <- systematic tile t
  int lost[kMaxCode];
  int tuse[kMaxCode];          // code tiles read, ascending: surviving systematic, used checksum
  int nuse;
  int bad;
};

// Every thread of the CTA (nthr threads, index tid) calls it; false when G^ is singular (then
// status gets CQR_EUNRECOVERABLE when report is set).
template <typename T>
__device__ __forceinline__ bool decode_setup(const Geo& g, const DecodePlan& p,
                                             const double* __restrict__ Gt,
                                             const double* __restrict__ Gh, DecodeScratch<T>& sh,
                                             int tid, int nthr, int* status, bool report) {
  const bool isQ = (p.kind == 0);
  const int nsys = p.nsys, f = g.f, f1 = p.f1, f2 = p.f2;
  auto gen = [&](int i, int t) -> double { return isQ ? Gt[i * g.p_r + t] : Gh[t * f + i]; };
  if (tid == 0) {
    sh.bad = 0;
    for (int t = 0; t < nsys + f; ++t) sh.lost[t] = 0;
    for (int b = 0; b < f1; ++b) sh.lost[p.A_fail[b]] = 1;
    for (int e = 0; e < f2; ++e) sh.lost[nsys + p.C_fail[e]] = 1;
    int nu = 0;
    for (int t = 0; t < nsys + f; ++t) {
      if (sh.lost[t]) continue;
      bool used = (t < nsys);
      if (!used)
        for (int u = 0; u < f1; ++u) used |= (p.C_use[u] == t - nsys);
      if (used) sh.tuse[nu++] = t;
    }
    sh.nuse = nu;
    // G^ = G~[C_use, A_fail]; invert by Gauss-Jordan (Golub & Van Loan 3.4), FP64
    for (int r = 0; r < f1; ++r)
      for (int q = 0; q < 2 * f1; ++q)
        sh.a[r][q] = (q < f1) ? gen(p.C_use[r], p.A_fail[q]) : (q - f1 == r ? 1.0 : 0.0);
    for (int col = 0; col < f1 && !sh.bad; ++col) {
      int piv = col;
      for (int r = col + 1; r < f1; ++r)
        if (fabs(sh.a[r][col]) > fabs(sh.a[piv][col])) piv = r;
      if (!(fabs(sh.a[piv][col]) > 0.0)) {
        sh.bad = 1;
        break;
      }
      if (piv != col)
        for (int q = 0; q < 2 * f1; ++q) {
          const double t = sh.a[col][q];
          sh.a[col][q] = sh.a[piv][q];
          sh.a[piv][q] = t;
        }
      const double pv = sh.a[col][col];
      for (int q = 0; q < 2 * f1; ++q) sh.a[col][q] = sh.a[col][q] / pv;
      for (int r = 0; r < f1; ++r) {
        if (r == col) continue;
        const double fc = sh.a[r][col];
        if (fc != 0.0)
          for (int q = 0; q < 2 * f1; ++q) sh.a[r][q] -= fc * sh.a[col][q];
      }
    }
    for (int r = 0; r < f1; ++r)
      for (int q = 0; q < f1; ++q) sh.Ginv[r * kMaxF + q] = sh.a[r][f1 + q];
    if (sh.bad && report) set_status(status, CQR_EUNRECOVERABLE, p.idx);
  }
  __syncthreads();
  if (sh.bad) return false;
  for (int idx = tid; idx < f1 * (nsys + f); idx += nthr) {
    const int b = idx / (nsys + f), t = idx % (nsys + f);
    double cv = 0.0;
    if (t < nsys) {
      if (!sh.lost[t])
        for (int u = 0; u < f1; ++u) cv -= sh.Ginv[b * kMaxF + u] * gen(p.C_use[u], t);
    } else {
      for (int u = 0; u < f1; ++u)
        if (p.C_use[u] == t - nsys) cv = sh.Ginv[b * kMaxF + u];
    }
    sh.coef[b][t] = (T)cv;
  }
  for (int idx = tid; idx < f2 * nsys; idx += nthr) {
    const int e = idx / nsys, t = idx % nsys;
    sh.cenc[e][t] = (T)gen(p.C_fail[e], t);
  }
  __syncthreads();
  return true;
}

// Position (r, s) of the code's tiles: r < mb (Q) or nb (R) within a tile, s < nb.  The code
// tiles are read U at a time (U independent loads in flight per thread) and summed in
// ascending order whatever U is, so every U gives the same bits.
template <typename T, int U = 1>
__device__ __forceinline__ void decode_apply(const Geo& g, const DecodePlan& p,
                                             const DecodeScratch<T>& sh, T* Q, T* R, int64_t r,
                                             int64_t s) {
  const bool isQ = (p.kind == 0);
  const int nsys = p.nsys, f1 = p.f1, f2 = p.f2;
  T* base = isQ ? Q + (int64_t)p.idx * g.nb * g.ldq : R + (int64_t)p.idx * g.nb;
  const int64_t tstride = isQ ? g.mb : g.nb * g.ldr;
  const int64_t ld = isQ ? g.ldq : g.ldr;
  T* ptr = base + r + s * ld;
  T xb[kMaxF], ce[kMaxF];
#pragma unroll
  for (int k = 0; k < kMaxF; ++k) {
    xb[k] = T(0);
    ce[k] = T(0);
  }
  auto add = [&](int t, T val) {
#pragma unroll
    for (int b = 0; b < kMaxF; ++b)
      if (b < f1) xb[b] += sh.coef[b][t] * val;
    if (t < nsys) {
#pragma unroll
      for (int e = 0; e < kMaxF; ++e)
        if (e < f2) ce[e] += sh.cenc[e][t] * val;
    }
  };
  if constexpr (U == 1) {
    for (int u = 0; u < sh.nuse; ++u) {
      const int t = sh.tuse[u];
      add(t, ptr[(int64_t)t * tstride]);
    }
  } else {
    for (int u0 = 0; u0 < sh.nuse; u0 += U) {
      int tt[U];
      T v[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        tt[k] = (u0 + k < sh.nuse) ? sh.tuse[u0 + k] : -1;
        v[k] = tt[k] >= 0 ? ptr[(int64_t)tt[k] * tstride] : T(0);
      }
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (tt[k] >= 0) add(tt[k], v[k]);
    }
  }
#pragma unroll
  for (int b = 0; b < kMaxF; ++b)
    if (b < f1) {
      ptr[(int64_t)p.A_fail[b] * tstride] = xb[b];
#pragma unroll
      for (int e = 0; e < kMaxF; ++e)
        if (e < f2) ce[e] += sh.cenc[e][p.A_fail[b]] * xb[b];
    }
#pragma unroll
  for (int e = 0; e < kMaxF; ++e)
    if (e < f2) ptr[(int64_t)(nsys + p.C_fail[e]) * tstride] = ce[e];
}

// The arithmetic of the four-row FP32 decode on values supplied by fetch(u), the float4 of
// code tile tuse[u] at the position; the rebuilt tiles are stored through ptr (tile k at
// ptr + k * tstride, 16-byte aligned).  Every element is summed in the same order as
// decode_apply, so the result has the same bits whatever supplies the values.
template <int UG = 4, typename Fetch>
__device__ __forceinline__ void decode_combine4(const DecodePlan& p,
                                                const DecodeScratch<float>& sh, float* ptr,
                                                int64_t tstride, Fetch fetch) {
  constexpr int NF = 4;
  const int nsys = p.nsys, f1 = p.f1, f2 = p.f2;
  float4 xb[NF], ce[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    xb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    ce[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  auto fma4 = [](float4& acc, float c, const float4& v) {
    acc.x += c * v.x;
    acc.y += c * v.y;
    acc.z += c * v.z;
    acc.w += c * v.w;
  };
  auto add = [&](int t, const float4& val) {
#pragma unroll
    for (int b = 0; b < NF; ++b)
      if (b < f1) fma4(xb[b], sh.coef[b][t], val);
    if (t < nsys) {
#pragma unroll
      for (int e = 0; e < NF; ++e)
        if (e < f2) fma4(ce[e], sh.cenc[e][t], val);
    }
  };
  for (int u0 = 0; u0 < sh.nuse; u0 += UG) {  // UG tile loads in flight
    int tt[UG];
    float4 v[UG];
#pragma unroll
    for (int k = 0; k < UG; ++k) {
      tt[k] = (u0 + k < sh.nuse) ? sh.tuse[u0 + k] : -1;
      v[k] = tt[k] >= 0 ? fetch(u0 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < UG; ++k)
      if (tt[k] >= 0) add(tt[k], v[k]);
  }
#pragma unroll
  for (int b = 0; b < NF; ++b)
    if (b < f1) {
      *reinterpret_cast<float4*>(ptr + (int64_t)p.A_fail[b] * tstride) = xb[b];
#pragma unroll
      for (int e = 0; e < NF; ++e)
        if (e < f2) fma4(ce[e], sh.cenc[e][p.A_fail[b]], xb[b]);
    }
#pragma unroll
  for (int e = 0; e < NF; ++e)
    if (e < f2) *reinterpret_cast<float4*>(ptr + (int64_t)(nsys + p.C_fail[e]) * tstride) = ce[e];
}

// Four consecutive rows r4 .. r4+3 of position column s in one thread, FP32, with 16-byte
// loads and stores (a warp reads 512 contiguous bytes of each code tile, eight tiles in
// flight); f <= 4.  The
// caller guarantees 16-byte alignment: the tile height and the leading dimension are
// multiples of four and r4 is.
__device__ __forceinline__ void decode_apply4(const Geo& g, const DecodePlan& p,
                                              const DecodeScratch<float>& sh, float* Q, float* R,
                                              int64_t r4, int64_t s) {
  const bool isQ = (p.kind == 0);
  float* base = isQ ? Q + (int64_t)p.idx * g.nb * g.ldq : R + (int64_t)p.idx * g.nb;
  const int64_t tstride = isQ ? g.mb : g.nb * g.ldr;
  const int64_t ld = isQ ? g.ldq : g.ldr;
  float* ptr = base + r4 + s * ld;
  decode_combine4<8>(p, sh, ptr, tstride, [&](int u) {
    return *reinterpret_cast<const float4*>(ptr + (int64_t)sh.tuse[u] * tstride);
  });
}

}  // namespace cqr

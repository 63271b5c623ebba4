// Persistent form of the block-speculative G-space iterations: one
// cooperative launch runs every iteration of the power iteration
// (Algorithm 1) and of the first doubling step (k = 2) of the simultaneous
// iteration (Algorithm 2) for all rows of a block.
//
// Within a block with no event, row t of the block sees the leading
// m_t = r0 + t + 1 rows of the buffer, i.e. the leading m_t x m_t principal
// submatrix of the block's Gram G.  Every column of the batch matrix belongs
// to one row t, is zero below m_t, and is multiplied by G each iteration.
//
// Work split.  CTA b owns the 16-row tiles b, b + grid, ... of every product
// Y = G X; when it owns a single tile, its 16 rows of G stay in shared memory
// for the whole launch.  Each iteration
//   (1) reduces the previous iteration's per-CTA partial sums, in a fixed
//       order, into the normalisation coefficients of every column;
//   (2) forms X_old = Y_old * coefficients while loading Y_old (X_old is
//       never stored) and computes its rows of Y_new = G X_old;
//   (3) writes its rows of Y_new and its partial sums;
//   (4) waits at a grid barrier (bounded: a wait that gives up sets
//       AS_ETIMEOUT in the status word and every CTA returns).
// Y and the partial sums are double buffered, so one barrier per iteration
// suffices: a CTA can only overwrite a buffer after every CTA has passed the
// barrier that follows its last read of it.
//
// Normalisation.  Power-iteration columns are scaled by 1/||y|| (Algorithm 1
// iterates the direction).  Each simultaneous-iteration pair is
// orthonormalised through the Cholesky factor of its 2 x 2 Gram; this keeps
// the span, and the final Rayleigh-Ritz step is exact for any basis of it.
// Per-element arithmetic is FP32 (FP64 throughput is a small fraction of
// FP32 on this part); the final sums (sigma^2 and the 2 x 2 Rayleigh-Ritz
// data) are reduced over the CTAs in FP64.
//
// Column layout (column-major, leading dimension ldy): power-iteration
// columns 0 .. 2*npi-1 (npi = ceil(nb/2), one zero padding column when nb is
// odd), then the pair of row t at columns 2*npi + 2t and 2*npi + 2t + 1.
#include <algorithm>
#include <mutex>

#include "grid.cuh"
#include "kernels.cuh"

namespace as {

namespace {

constexpr int kTile = 16;            // rows of G per CTA tile
constexpr int kPThreads = 256;
constexpr int kPWarps = kPThreads / 32;
constexpr int kPairsPerUnit = 4;     // a warp unit: 4 column pairs (8 columns) x one K range
constexpr int kMaxUnits = 64;
constexpr int kSlots = 6;            // partial sums per pair
constexpr int kMaxGrid = 1024;
constexpr int kMaxGroup = 32;        // problems in one grouped launch

struct PersistArgs {
  const float* G;      // FP32 copy of the leading mmax x mmax block of G (row-major, ld ldg)
  long long ldg;
  int mmax;
  float* Y;            // two buffers of ybuf floats: columns of ldy floats
  long long ybuf;
  int ldy;
  float* X;            // out: the final basis of every pair (ld ldx)
  int ldx;
  float* part;         // two buffers of pbuf floats: [pair * kSlots + slot][cta]
  long long pbuf;
  unsigned* cnt;       // barrier arrivals (zero at launch)
  int* status;
  int nb, npi, r0, k_pi, q;
  int ntiles;
  double* sig2;        // nb
  double* ritz;        // 2 nb
};

// Rows in use by column c (zero for the padding column).
__device__ __forceinline__ int col_rows(const PersistArgs& a, int c) {
  const int pcol = 2 * a.npi;
  if (c < pcol) return (c < a.nb) ? a.r0 + c + 1 : 0;
  return a.r0 + ((c - pcol) >> 1) + 1;
}

// K splits per column group so that the units spread evenly over the warps.
__device__ __forceinline__ int pick_ksplit(int ngrp) {
  int best = 1;
  float bc = 1e30f;
  for (int ks = 1; ks <= 8; ++ks) {
    if (ngrp * ks > kMaxUnits) break;
    const float c = (float)((ngrp * ks + kPWarps - 1) / kPWarps) / (float)ks;
    if (c < bc * (1.f - 1e-6f)) { bc = c; best = ks; }
  }
  return best;
}

// Sums v[0..128) over the 32 lanes by recursive halving: 124 shuffles, after
// which lane L holds the totals of entries 4L .. 4L+3 in v[0..4).
template <int H>
__device__ __forceinline__ void halve_step(float (&v)[128], int lane) {
  constexpr int o = H / 4;   // partner distance: 16, 8, 4, 2, 1 for H = 64 .. 4
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float send = up ? v[i] : v[i + H];
    const float keep = up ? v[i + H] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

__device__ __forceinline__ void warp_transpose_sum128(float (&v)[128], int lane) {
  halve_step<64>(v, lane);
  halve_step<32>(v, lane);
  halve_step<16>(v, lane);
  halve_step<8>(v, lane);
  halve_step<4>(v, lane);
}

__device__ __forceinline__ void eig2_sym(double s00, double s01, double s11, double& l0, double& l1, double& v00,
                                         double& v01, double& v10, double& v11) {
  const double tr = 0.5 * (s00 + s11), df = 0.5 * (s00 - s11);
  const double rad = sqrt(df * df + s01 * s01);
  l0 = tr + rad;
  l1 = tr - rad;
  if (rad == 0.0) { v00 = 1; v10 = 0; v01 = 0; v11 = 1; return; }
  const double th = 0.5 * atan2(2.0 * s01, s00 - s11);
  v00 = cos(th); v10 = sin(th); v01 = -v10; v11 = v00;
}

// Shared memory (floats): [Gs: kTile x mpad, GSMEM only] [coef: 4 per pair]
// [red: kMaxUnits x 128] [Ys: 2 * pairs x kTile].
// The body of one problem: G CTAs (this one is blk of them) iterate to
// `iters` (at least the problem's own max(k_pi, q); a grouped launch runs to
// the largest of its problems and a problem idles past its own), meeting the
// other CTAs of the launch (gtotal in all) at each grid barrier.
template <bool GSMEM>
__device__ __forceinline__ void persist_body(const PersistArgs& a, const int G, const int blk, const int iters,
                                             const unsigned gtotal) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = a.npi + a.nb;
  const int mpad = (a.mmax + 3) & ~3;
  float* Gs = sm;
  float* coef = sm + (GSMEM ? kTile * mpad : 0);
  float* red = coef + 4 * ((P + 3) & ~3);
  float* Ys = red + kMaxUnits * 128;

  if (GSMEM) {   // this CTA owns exactly one tile
    const int row0 = blk * kTile;
    const int R = min(kTile, a.mmax - row0);
    for (int e = tid; e < kTile * mpad; e += kPThreads) {
      const int r = e / mpad, k = e - r * mpad;
      Gs[e] = (r < R && k < a.mmax) ? a.G[(size_t)(row0 + r) * a.ldg + k] : 0.f;
    }
  }
  for (int it = 0; it <= iters; ++it) {
    const bool pi_on = it <= a.k_pi, si_on = it <= a.q;
    const int pa0 = pi_on ? 0 : a.npi, pa1 = si_on ? P : a.npi;
    const int nact = pa1 - pa0;
    const float* Yold = a.Y + (size_t)((it + 1) & 1) * a.ybuf;
    float* Ynew = a.Y + (size_t)(it & 1) * a.ybuf;
    const float* pold = a.part + (size_t)((it + 1) & 1) * a.pbuf;
    float* pnew = a.part + (size_t)(it & 1) * a.pbuf;

    // product geometry: units of 4 pairs x one of KS ranges of kc rows of X
    const int ngrp = (nact + kPairsPerUnit - 1) / kPairsPerUnit;
    const int KS = pick_ksplit(ngrp);
    const int nunits = ngrp * KS;
    const int kc = ((a.mmax + KS - 1) / KS + 127) / 128 * 128;
    // unit u covers pairs [pb, pb + nv) and rows [k0, k1) of X_old
    auto unit_of = [&](int uu, int& pb, int& nv, int& k0, int& k1) {
      const int gi = uu / KS, ks = uu - gi * KS;
      pb = pa0 + gi * kPairsPerUnit;
      nv = min(kPairsPerUnit, pa1 - pb);
      k0 = ks * kc;
      k1 = min(a.mmax, k0 + kc);
    };
    // raw Y_old rows k .. k+3 (k = kk + 4 lane) of the unit's 8 columns
    // (k0 and interior k1 are multiples of 128; only k1 = mmax can cut a quad)
    auto load = [&](float4 (&v)[2 * kPairsPerUnit], int pb, int nv, int kk, int k1) {
      const float* ybase = Yold + (size_t)(2 * pb) * a.ldy;
      const int k = kk + 4 * lane;
#pragma unroll
      for (int j = 0; j < 2 * kPairsPerUnit; ++j) {
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((j >> 1) < nv && k < k1) {
          const float* q = ybase + (size_t)j * a.ldy + k;
          if (k + 3 < k1) {
            v[j] = __ldcg(reinterpret_cast<const float4*>(q));
          } else {
            v[j].x = __ldcg(q);
            if (k + 1 < k1) v[j].y = __ldcg(q + 1);
            if (k + 2 < k1) v[j].z = __ldcg(q + 2);
          }
        }
      }
    };
    // the warp's first item is the same for every tile: its loads go out now,
    // while the coefficient phase waits on the partial sums
    float4 yn[2 * kPairsPerUnit];
    bool have = false;
    if (warp < nunits) {
      int pb, nv, k0, k1;
      unit_of(warp, pb, nv, k0, k1);
      if (k0 < k1) { load(yn, pb, nv, k0, k1); have = true; }
    }

    // (1) coefficients: x0 = c00 y0 + c10 y1, x1 = c01 y0 + c11 y1
    if (it == 0) {
      for (int p = tid; p < P; p += kPThreads) {
        coef[4 * p] = 1.f; coef[4 * p + 1] = 0.f; coef[4 * p + 2] = 0.f; coef[4 * p + 3] = 1.f;
      }
    } else {
      // a warp takes 4 pairs at a time so that all their loads are in flight together
      for (int pbase = pa0 + 4 * warp; pbase < pa1; pbase += 4 * kPWarps) {
        float sv[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) sv[j][0] = sv[j][1] = sv[j][2] = 0.f;
        // all loads of a chunk of 4 x 32 CTAs are issued before any add uses
        // them (in-order issue would otherwise pay one L2 round trip per 32)
        for (int g0 = 0; g0 < G; g0 += 128) {
          float buf[4][4][3];
#pragma unroll
          for (int gg = 0; gg < 4; ++gg) {
            const int g = g0 + 32 * gg + lane;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int p = pbase + j;
              const bool on = p < pa1 && g < G;
              const float* q0 = pold + (size_t)(p * kSlots) * G + g;
              buf[gg][j][0] = on ? __ldcg(q0) : 0.f;
              buf[gg][j][1] = on ? __ldcg(q0 + G) : 0.f;
              buf[gg][j][2] = (on && p >= a.npi) ? __ldcg(q0 + 2 * G) : 0.f;
            }
          }
#pragma unroll
          for (int gg = 0; gg < 4; ++gg)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              sv[j][0] += buf[gg][j][0];
              sv[j][1] += buf[gg][j][1];
              sv[j][2] += buf[gg][j][2];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          sv[j][0] = warp_sum(sv[j][0]);
          sv[j][1] = warp_sum(sv[j][1]);
          sv[j][2] = warp_sum(sv[j][2]);
        }
        const int p = pbase + lane;
        if (lane < 4 && p < pa1) {
          float s0 = sv[0][0], s1 = sv[0][1], s2 = sv[0][2];
#pragma unroll
          for (int j = 1; j < 4; ++j)
            if (lane == j) { s0 = sv[j][0]; s1 = sv[j][1]; s2 = sv[j][2]; }
          float c00 = 0.f, c10 = 0.f, c01 = 0.f, c11 = 0.f;
          if (p < a.npi) {
            c00 = (s0 > 0.f) ? rsqrtf(s0) : 0.f;
            c11 = (s1 > 0.f) ? rsqrtf(s1) : 0.f;
          } else if (s0 > 0.f) {
            // [y0 y1] = [x0 x1] R, R = [[sqrt(a), b/sqrt(a)], [0, sqrt(c - b^2/a)]]
            const float r00 = sqrtf(s0), l = s1 / s0;
            const float sc = fmaxf(s2 - s1 * l, 1e-12f * s2);
            c00 = 1.f / r00;
            if (s2 > 0.f) {
              c11 = rsqrtf(sc);
              c01 = -l * c11;
            }
          }
          coef[4 * p] = c00; coef[4 * p + 1] = c10; coef[4 * p + 2] = c01; coef[4 * p + 3] = c11;
        }
      }
    }
    __syncthreads();

    // (2)-(3) rows of Y_new = G X_old for this CTA's tiles
    float ps[kSlots] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int tile = blk; tile < a.ntiles; tile += G) {
      const int row0 = tile * kTile;
      const int R = min(kTile, a.mmax - row0);
      // items (unit, 128-row step) in order; the next item's loads are issued
      // before the current item's arithmetic, across unit boundaries
      for (int u = warp; u < nunits; u += kPWarps) {
        int pb, nv, k0, k1;
        unit_of(u, pb, nv, k0, k1);
        const float4* cf4 = reinterpret_cast<const float4*>(coef) + pb;   // (c00, c10, c01, c11) per pair
        if (!have && k0 < k1) load(yn, pb, nv, k0, k1);
        have = false;
        float acc[128];
#pragma unroll
        for (int e = 0; e < 128; ++e) acc[e] = 0.f;
        float4 yv[2 * kPairsPerUnit];
        for (int kk = k0; kk < k1; kk += 128) {
          // X_old = Y_old * coefficients (pairs past nv are zero)
#pragma unroll
          for (int j = 0; j < kPairsPerUnit; ++j) {
            const float4 c = cf4[j < nv ? j : 0];
            const float4 ya = yn[2 * j], yb = yn[2 * j + 1];
            yv[2 * j] = make_float4(fmaf(c.x, ya.x, c.y * yb.x), fmaf(c.x, ya.y, c.y * yb.y),
                                    fmaf(c.x, ya.z, c.y * yb.z), fmaf(c.x, ya.w, c.y * yb.w));
            yv[2 * j + 1] = make_float4(fmaf(c.z, ya.x, c.w * yb.x), fmaf(c.z, ya.y, c.w * yb.y),
                                        fmaf(c.z, ya.z, c.w * yb.z), fmaf(c.z, ya.w, c.w * yb.w));
          }
          if (kk + 128 < k1) {
            load(yn, pb, nv, kk + 128, k1);
          } else if (u + kPWarps < nunits) {   // first step of the warp's next unit
            int pb2, nv2, k02, k12;
            unit_of(u + kPWarps, pb2, nv2, k02, k12);
            if (k02 < k12) { load(yn, pb2, nv2, k02, k12); have = true; }
          }
          const int k = kk + 4 * lane;
#pragma unroll
          for (int r = 0; r < kTile; ++r) {
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (GSMEM) {
              if (k < k1) g = *reinterpret_cast<const float4*>(Gs + r * mpad + k);
            } else if (r < R && k < k1) {
              const float* gp = a.G + (size_t)(row0 + r) * a.ldg + k;
              g.x = __ldg(gp);
              if (k + 1 < k1) g.y = __ldg(gp + 1);
              if (k + 2 < k1) g.z = __ldg(gp + 2);
              if (k + 3 < k1) g.w = __ldg(gp + 3);
            }
#pragma unroll
            for (int j = 0; j < 2 * kPairsPerUnit; ++j) {
              float t = acc[j * kTile + r];
              t = fmaf(g.x, yv[j].x, t);
              t = fmaf(g.y, yv[j].y, t);
              t = fmaf(g.z, yv[j].z, t);
              t = fmaf(g.w, yv[j].w, t);
              acc[j * kTile + r] = t;
            }
          }
        }
        warp_transpose_sum128(acc, lane);
        reinterpret_cast<float4*>(red + (size_t)u * 128)[lane] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      }
      __syncthreads();
      // combine the K splits in order; Ys[local column][row], local column = column - 2*pa0
      for (int o = tid; o < ngrp * 128; o += kPThreads) {
        const int gi = o >> 7, idx = o & 127;
        float v = 0.f;
        for (int ks = 0; ks < KS; ++ks) v += red[(size_t)(gi * KS + ks) * 128 + idx];
        const int cl = gi * 2 * kPairsPerUnit + (idx >> 4), r = idx & 15;
        if (cl < 2 * nact) Ys[cl * kTile + r] = v;
      }
      __syncthreads();
      for (int o = tid; o < 2 * nact * kTile; o += kPThreads) {
        const int cl = o / kTile, r = o - cl * kTile;
        const int c = 2 * pa0 + cl, row = row0 + r;
        const float v = (r < R && row < col_rows(a, c)) ? Ys[o] : 0.f;
        Ys[o] = v;
        if (r < R) Ynew[(size_t)c * a.ldy + row] = v;
      }
      __syncthreads();
      if (tid < nact) {
        const int p = pa0 + tid;
        const bool si = p >= a.npi;
        const bool fin = si ? (it == a.q) : (it == a.k_pi);
        const float* y0 = Ys + (2 * tid) * kTile;
        const float* y1 = y0 + kTile;
        if (!fin) {
          for (int r = 0; r < R; ++r) {
            ps[0] = fmaf(y0[r], y0[r], ps[0]);
            if (si) {
              ps[1] = fmaf(y0[r], y1[r], ps[1]);
              ps[2] = fmaf(y1[r], y1[r], ps[2]);
            } else {
              ps[1] = fmaf(y1[r], y1[r], ps[1]);
            }
          }
        } else {
          const float c00 = coef[4 * p], c10 = coef[4 * p + 1], c01 = coef[4 * p + 2], c11 = coef[4 * p + 3];
          const float* o0 = Yold + (size_t)(2 * p) * a.ldy + row0;
          const float* o1 = o0 + a.ldy;
          for (int r = 0; r < R; ++r) {
            const float ya = __ldcg(o0 + r), yb = __ldcg(o1 + r);
            const float x0 = fmaf(c00, ya, c10 * yb), x1 = fmaf(c01, ya, c11 * yb);
            if (!si) {
              ps[0] = fmaf(x0, y0[r], ps[0]);
              ps[1] = fmaf(x1, y1[r], ps[1]);
            } else {
              ps[0] = fmaf(x0, y0[r], ps[0]);
              ps[1] = fmaf(0.5f, fmaf(x0, y1[r], x1 * y0[r]), ps[1]);
              ps[2] = fmaf(x1, y1[r], ps[2]);
              ps[3] = fmaf(y0[r], y0[r], ps[3]);
              ps[4] = fmaf(y0[r], y1[r], ps[4]);
              ps[5] = fmaf(y1[r], y1[r], ps[5]);
              a.X[(size_t)(2 * p) * a.ldx + row0 + r] = x0;
              a.X[(size_t)(2 * p + 1) * a.ldx + row0 + r] = x1;
            }
          }
        }
      }
      __syncthreads();
    }
    if (tid < nact) {
      const int p = pa0 + tid;
#pragma unroll
      for (int e = 0; e < kSlots; ++e) pnew[(size_t)(p * kSlots + e) * G + blk] = ps[e];
    }
    if (!grid_barrier(a.cnt, (unsigned)(it + 1) * gtotal, a.status)) return;

    // final values (FP64 over the CTAs), spread over the CTAs
    if (pi_on && it == a.k_pi && warp == 0) {
      for (int t = blk; t < a.nb; t += G) {
        const float* q0 = pnew + (size_t)((t >> 1) * kSlots + (t & 1)) * G;
        double s = 0.0;
        for (int g = lane; g < G; g += 32) s += (double)__ldcg(q0 + g);
        s = warp_sum(s);
        if (lane == 0) a.sig2[t] = s;
      }
    }
    if (si_on && it == a.q && warp == 1) {
      for (int t = blk; t < a.nb; t += G) {
        const float* q0 = pnew + (size_t)((a.npi + t) * kSlots) * G;
        double v[kSlots];
#pragma unroll
        for (int e = 0; e < kSlots; ++e) {
          double s = 0.0;
          for (int g = lane; g < G; g += 32) s += (double)__ldcg(q0 + (size_t)e * G + g);
          v[e] = warp_sum(s);
        }
        if (lane == 0) {
          // S = X^T G X, H = (G X)^T (G X); G-orthonormal W = X V diag(a),
          // Ritz values = eig(diag(a) V^T H V diag(a))
          double l0, l1, v00, v01, v10, v11;
          eig2_sym(v[0], v[1], v[2], l0, l1, v00, v01, v10, v11);
          const double tol = 1e-6 * fmax(l0, 0.0);
          const double a0 = (l0 > tol && l0 > 0) ? 1.0 / sqrt(l0) : 0.0;
          const double a1 = (l1 > tol && l1 > 0) ? 1.0 / sqrt(l1) : 0.0;
          const double h00 = v[3], h01 = v[4], h11 = v[5];
          const double hv00 = h00 * v00 + h01 * v10, hv10 = h01 * v00 + h11 * v10;
          const double hv01 = h00 * v01 + h01 * v11, hv11 = h01 * v01 + h11 * v11;
          const double m00 = a0 * a0 * (v00 * hv00 + v10 * hv10);
          const double m01 = a0 * a1 * (v00 * hv01 + v10 * hv11);
          const double m11 = a1 * a1 * (v01 * hv01 + v11 * hv11);
          const double tr = 0.5 * (m00 + m11), df = 0.5 * (m00 - m11);
          const double rad = sqrt(df * df + m01 * m01);
          a.ritz[2 * t] = (a0 > 0) ? tr + rad : 0.0;
          a.ritz[2 * t + 1] = (a0 > 0 && a1 > 0) ? tr - rad : 0.0;
        }
      }
    }
  }
}

template <bool GSMEM>
__global__ void __launch_bounds__(kPThreads, 1) batch_persist_kernel(const PersistArgs a) {
  persist_body<GSMEM>(a, gridDim.x, blockIdx.x, max(a.k_pi, a.q), gridDim.x);
}

// Many sketches' blocks in one cooperative launch: problem j owns CTAs
// [cta0[j], cta0[j+1]), one 16-row tile each with its rows of G in shared
// memory (the same CTAs and arithmetic as its own launch, so its results are
// bitwise those of running it alone); every CTA meets all others at the
// shared grid barrier.
struct GroupArgs {
  PersistArgs p[kMaxGroup];
  int cta0[kMaxGroup + 1];
  int n;
  int iters;
};

__global__ void __launch_bounds__(kPThreads, 1) batch_group_kernel(const __grid_constant__ GroupArgs g) {
  int j = 0;
  while (j + 1 < g.n && (int)blockIdx.x >= g.cta0[j + 1]) ++j;
  persist_body<true>(g.p[j], g.cta0[j + 1] - g.cta0[j], (int)blockIdx.x - g.cta0[j], g.iters, gridDim.x);
}

// Starting vectors (buffer 1 = the buffer iteration 0 reads): x^(0) of row t
// (Philox purpose 3, counter (3, i0 + t, 0, e >> 2)) in column t, and the
// test matrix Pi (n2 x 2 row-major, purpose 4, sub-index j = 1) of row t in
// its pair's columns; zero below m_t.  Grid (nb, 2, z): the z blocks of a
// column split its four-value Philox blocks (the FP64 Box-Muller transform is
// slow on this part, so a column is spread over several SMs).
__global__ void persist_fill_kernel(float* Y, int ldy, int mmax, int nb, int npi, int r0, Key key, uint64_t i0) {
  const int t = blockIdx.x, kind = blockIdx.y;
  const int m = r0 + t + 1;
  const uint64_t i = i0 + (uint64_t)t;
  if (kind == 0) {
    float* x = Y + (size_t)t * ldy;
    for (int blk = blockIdx.z * blockDim.x + threadIdx.x; blk * 4 < mmax; blk += blockDim.x * gridDim.z) {
      double z[4];
      gauss4(key, kPurposePiStart, i, 0, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int p = blk * 4 + l;
        if (p < mmax) x[p] = (p < m) ? (float)z[l] : 0.f;
      }
    }
    if (t == nb - 1 && (nb & 1)) {   // padding column of the last power-iteration pair
      float* z = Y + (size_t)nb * ldy;
      for (int p = blockIdx.z * blockDim.x + threadIdx.x; p < mmax; p += blockDim.x * gridDim.z) z[p] = 0.f;
    }
  } else {
    float* x0 = Y + (size_t)(2 * npi + 2 * t) * ldy;
    for (int blk = blockIdx.z * blockDim.x + threadIdx.x; blk * 4 < 2 * mmax; blk += blockDim.x * gridDim.z) {
      double z[4];
      gauss4(key, kPurposeSiTest, i, 1, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int e = blk * 4 + l;
        if (e < 2 * mmax) {
          const int p = e >> 1, c = e & 1;
          x0[(size_t)c * ldy + p] = (p < m) ? (float)z[l] : 0.f;
        }
      }
    }
  }
}

struct PersistDevice {
  int sms = 0;
  int optin = 0;                   // opt-in shared memory per block
  int stat[2] = {-1, -1};          // static shared memory of each variant
  size_t attr[2] = {0, 0};         // dynamic shared memory limit set so far
  int gstat = 0;                   // the grouped kernel's static shared memory
  size_t gattr = 0;                // and its dynamic limit set so far
};
PersistDevice g_pdev[64];
std::mutex g_pdev_mu;   // guards g_pdev (sketches may run from several host threads)

size_t persist_smem_bytes(bool gsmem, int mmax, int P) {
  const size_t mpad = (size_t)((mmax + 3) & ~3);
  return sizeof(float) * ((gsmem ? kTile * mpad : 0) + 4 * (size_t)((P + 3) & ~3) + (size_t)kMaxUnits * 128 +
                          (size_t)2 * P * kTile);
}

}  // namespace

int batch_si_col(int nb, int t) { return 2 * ((nb + 1) / 2) + 2 * t; }

size_t batch_persist_ycols(int bmax) { return 2 * (size_t)((bmax + 1) / 2) + 2 * (size_t)bmax; }

size_t batch_persist_part_floats(int bmax) {
  return 2 * (size_t)kSlots * ((bmax + 1) / 2 + bmax) * kMaxGrid;
}

void launch_persist_fill(cudaStream_t s, const PersistBuffers& pb, int mmax, int nb, int npi, int r0, Key key,
                         uint64_t i0) {
  const int zc = std::max(1, (2 * mmax / 4 + 127) / 128);
  persist_fill_kernel<<<dim3(nb, 2, zc), 128, 0, s>>>(pb.Y + pb.ybuf, pb.ldy, mmax, nb, npi, r0, key, i0);
  count_launches(1);
}

int batch_group_capacity() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 0; }
  std::lock_guard<std::mutex> lk(g_pdev_mu);
  PersistDevice& pd = g_pdev[dev];
  if (pd.sms == 0 && cudaDeviceGetAttribute(&pd.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return pd.sms;   // one CTA per SM (255 registers x 256 threads)
}

int batch_group_tiles(const BatchJob& j) {
  const int mmax = j.r0 + j.nb;
  if (j.nb <= 0 || mmax > j.n2 || (size_t)2 * ((j.nb + 1) / 2 + j.nb) > j.pb.ycols || j.nb > j.pb.bmax) return 0;
  return (mmax + kTile - 1) / kTile;
}

as_status launch_batch_group(cudaStream_t s, const BatchJob* jobs, int n, unsigned* cnt) {
  if (n <= 0) return AS_OK;
  if (n > kMaxGroup) return AS_EINVAL;
  int dev = 0;
  AS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return AS_EINVAL;
  GroupArgs g{};
  size_t smax = 0;
  int total = 0, iters = 0;
  for (int j = 0; j < n; ++j) {
    const BatchJob& b = jobs[j];
    const int tiles = batch_group_tiles(b);
    if (tiles <= 0) return AS_EINVAL;
    const int mmax = b.r0 + b.nb, npi = (b.nb + 1) / 2, P = npi + b.nb;
    smax = std::max(smax, persist_smem_bytes(true, mmax, P));
    PersistArgs& a = g.p[j];
    a.G = b.Gf; a.ldg = b.n2; a.mmax = mmax;
    a.Y = b.pb.Y; a.ybuf = b.pb.ybuf; a.ldy = b.pb.ldy;
    a.X = b.pb.X; a.ldx = b.n2;
    a.part = b.pb.part; a.pbuf = (long long)kSlots * P * tiles;
    a.cnt = cnt; a.status = b.status;
    a.nb = b.nb; a.npi = npi; a.r0 = b.r0; a.k_pi = b.k_pi; a.q = b.q;
    a.ntiles = tiles;
    a.sig2 = b.pb.sig2; a.ritz = b.pb.ritz;
    g.cta0[j] = total;
    total += tiles;
    iters = std::max(iters, std::max(b.k_pi, b.q));
  }
  g.cta0[n] = total;
  g.n = n;
  g.iters = iters;
  {
    std::unique_lock<std::mutex> plk(g_pdev_mu);
    PersistDevice& pd = g_pdev[dev];
    if (pd.sms == 0) {
      AS_CUDA_TRY(cudaDeviceGetAttribute(&pd.sms, cudaDevAttrMultiProcessorCount, dev));
      AS_CUDA_TRY(cudaDeviceGetAttribute(&pd.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    }
    if (pd.optin == 0) AS_CUDA_TRY(cudaDeviceGetAttribute(&pd.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (pd.gattr == 0) {
      cudaFuncAttributes fa{};
      AS_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)batch_group_kernel));
      pd.gstat = (int)fa.sharedSizeBytes;
    }
    if (smax + (size_t)pd.gstat > (size_t)pd.optin) return AS_ENOTSUP;
    if (smax > pd.gattr) {
      AS_CUDA_TRY(cudaFuncSetAttribute((const void*)batch_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smax));
      pd.gattr = smax;
    }
    int per = 0;
    AS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_group_kernel, kPThreads, smax));
    if ((long long)per * pd.sms < total) return AS_ENOTSUP;
  }
  for (int j = 0; j < n; ++j) {
    const BatchJob& b = jobs[j];
    launch_persist_fill(s, b.pb, b.r0 + b.nb, b.nb, (b.nb + 1) / 2, b.r0, b.key, b.i0);
  }
  AS_CUDA_TRY(cudaGetLastError());
  AS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
  void* args[] = {&g};
  AS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)batch_group_kernel, dim3(total), dim3(kPThreads), args, smax, s));
  count_launches(1);
  return AS_OK;
}

as_status launch_batch_persist(cudaStream_t s, const float* Gf, int n2, int r0, int nb, int k_pi, int q, Key key,
                               uint64_t i0, const PersistBuffers& pb, int* status, Prof* prof) {
  if (nb <= 0) return AS_OK;
  const int mmax = r0 + nb;
  const int npi = (nb + 1) / 2, P = npi + nb;
  if (mmax > n2 || (size_t)2 * P > pb.ycols || nb > pb.bmax) return AS_EINVAL;
  int dev = 0;
  AS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return AS_EINVAL;
  std::unique_lock<std::mutex> plk(g_pdev_mu);
  PersistDevice& pd = g_pdev[dev];
  if (pd.sms == 0) {
    AS_CUDA_TRY(cudaDeviceGetAttribute(&pd.sms, cudaDevAttrMultiProcessorCount, dev));
    AS_CUDA_TRY(cudaDeviceGetAttribute(&pd.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (int v = 0; v < 2; ++v) {
      cudaFuncAttributes fa{};
      AS_CUDA_TRY(cudaFuncGetAttributes(&fa, v ? (const void*)batch_persist_kernel<true>
                                               : (const void*)batch_persist_kernel<false>));
      pd.stat[v] = (int)fa.sharedSizeBytes;
    }
  }
  // raise the variant's dynamic shared-memory limit to `bytes` (false: impossible)
  auto allow = [&](int v, size_t bytes) -> as_status {
    if (bytes + (size_t)pd.stat[v] > (size_t)pd.optin) return AS_ENOTSUP;
    if (bytes > pd.attr[v]) {
      AS_CUDA_TRY(cudaFuncSetAttribute(v ? (const void*)batch_persist_kernel<true>
                                         : (const void*)batch_persist_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      pd.attr[v] = bytes;
    }
    return AS_OK;
  };
  const int ntiles = (mmax + kTile - 1) / kTile;
  // one tile per CTA with G resident in shared memory when it fits and all
  // tiles can be co-resident; otherwise tiles loop over a co-resident grid
  bool gsmem = false;
  int grid = 0;
  size_t smem = persist_smem_bytes(true, mmax, P);
  if (allow(1, smem) == AS_OK) {
    int per = 0;
    AS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_persist_kernel<true>, kPThreads, smem));
    if ((long long)per * pd.sms >= ntiles) { gsmem = true; grid = ntiles; }
  }
  if (!gsmem) {
    smem = persist_smem_bytes(false, mmax, P);
    as_status st = allow(0, smem);
    if (st != AS_OK) return st;
    int per = 0;
    AS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_persist_kernel<false>, kPThreads, smem));
    if (per < 1) return AS_EDEVICE;
    grid = std::min(ntiles, per * pd.sms);
  }
  grid = std::min(grid, kMaxGrid);
  plk.unlock();

  if (prof) prof->begin(PK_BATCH_ORTH, s);
  launch_persist_fill(s, pb, mmax, nb, npi, r0, key, i0);
  AS_CUDA_TRY(cudaGetLastError());
  if (prof) prof->end(PK_BATCH_ORTH, s, 0.0, 12.0 * mmax * (double)nb);
  AS_CUDA_TRY(cudaMemsetAsync(pb.cnt, 0, sizeof(unsigned), s));
  PersistArgs a{};
  a.G = Gf; a.ldg = n2; a.mmax = mmax;
  a.Y = pb.Y; a.ybuf = pb.ybuf; a.ldy = pb.ldy;
  a.X = pb.X; a.ldx = n2;
  a.part = pb.part; a.pbuf = (long long)kSlots * P * grid;
  a.cnt = pb.cnt; a.status = status;
  a.nb = nb; a.npi = npi; a.r0 = r0; a.k_pi = k_pi; a.q = q;
  a.ntiles = ntiles;
  a.sig2 = pb.sig2; a.ritz = pb.ritz;
  void* args[] = {&a};
  if (prof) prof->begin(PK_BATCH_GEMM, s);
  AS_CUDA_TRY(cudaLaunchCooperativeKernel(gsmem ? (const void*)batch_persist_kernel<true>
                                                : (const void*)batch_persist_kernel<false>,
                                          dim3(grid), dim3(kPThreads), args, smem, s));
  count_launches(1);
  if (prof) {
    // algorithmic work: column c of row t is multiplied by the m_t x m_t block
    // (k_pi + 1 times for the power iteration, q + 1 times for each of the two
    // simultaneous-iteration columns); G read once, every column read and
    // written once per product
    double m2 = 0.0, m1 = 0.0;
    for (int t = 0; t < nb; ++t) {
      const double m = (double)(r0 + t + 1);
      m2 += m * m;
      m1 += m;
    }
    const double prods = (double)(k_pi + 1) + 2.0 * (double)(q + 1);
    // algorithmic work recorded at the block's decisions (add_work); issued here
    prof->end(PK_BATCH_GEMM, s, 0.0, 4.0 * (double)mmax * mmax + 8.0 * m1 * prods, 2.0 * m2 * prods);
  }
  return AS_OK;
}

}  // namespace as

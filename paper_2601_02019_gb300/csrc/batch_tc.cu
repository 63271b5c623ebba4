// Tensor-core form of the block-speculative G-space iterations (the tensor
// precision forms): the same power iteration (Algorithm 1) and first doubling
// step (k = 2) of the simultaneous iteration (Algorithm 2) for every row of a
// block as the FP32 persistent kernel, in one cooperative launch, with the
// products by G on tcgen05.
//
// Row t of the block sees the leading m_t = r0 + t + 1 rows of the buffer, so
// every column of the batch matrix is zero below m_t and each iteration is
//   Z = G Y_it,   Y_{it+1} = Z C_it   (rows >= m_t of each column zeroed),
// where C_it is the per-pair 2 x 2 normalisation of Y_it (1/||y|| for the
// power-iteration columns, the inverse Cholesky factor of the pair's Gram for
// a simultaneous-iteration pair).  G (C_it applied after the product) equals
// G (Y_it C_it) in exact arithmetic; applying it afterwards lets both operands
// of the product come from memory through TMA, in split-BF16 levels:
//   x = x0 + x1 (+ x2),  x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1),
// accumulating every level product whose order is above 2^-16 (three passes)
// or 2^-24 (six passes).
//
// Work split.  CTA (rb, ks) multiplies the 128 rows rb of G by the rows
// [ks kc, (ks+1) kc) of Y_it (UMMA M = 128, N = the padded column count,
// K = kc): a TMA producer lane streams, per 64-wide K tile, both BF16 levels
// of G and of Y (128-byte swizzle) through a 2-stage ring, one lane issues
// the three level products as tcgen05.mma into two TMEM accumulators (the
// leading level product and the corrections), and warps 4-7 (one TMEM lane
// quarter each) move the partial 128 x N block to global memory, after which
// warp 1 announces it to the row block.  Once the nks products of its row block are in, CTA
// (rb, ks) sums the K-split partials of its rpb rows of that row block in a
// fixed order, applies C_it, masks, writes Y_{it+1} (FP32 and its BF16
// levels) and its per-pair partial sums, and publishes them with a release
// flag (synchronisation below).  The coefficients C_it are computed from
// those partial sums by warps 2-7 (warps 4-7 after their epilogue, so the
// product's announcement never waits for the coefficients).  Every
// mbarrier, counter and flag wait is bounded; on a timeout the status word
// gets AS_ETIMEOUT and every CTA frees its TMEM and returns.
#include <algorithm>
#include <mutex>

#include "grid.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace as {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcStages = 2;   // ring stages; a stage holds one K tile of every level used
constexpr int kTcSlots = 6;     // partial sums per pair
constexpr int kTcMaxRpc = 32;   // rows per CTA in the reduction phase
constexpr int kTcMaxCols = 192; // batch columns (2 P)
constexpr int kTcMaxSplits = 16; // K ranges per row block (nks, checked at launch)

struct TcArgs {
  float* Y;            // FP32 columns, two buffers of ybuf floats, ld ldy
  long long ybuf;
  int ldy;
  __nv_bfloat16* Yb;   // BF16 levels: [level][buffer][ycols][ldyb]
  long long yblevel;   // elements per level (2 buffers)
  long long ybbuf;     // elements per buffer
  int ldyb;
  int ycols;
  float* X;            // final basis of every pair (ld ldx)
  int ldx;
  float* part;         // K-split partial products, two buffers of [nks][kpad][nc]
  long long pplane;
  float* sums;         // per-pair partial sums, two buffers of sbuf floats: [pair * kTcSlots + slot][cta]
  long long sbuf;
  unsigned* flags;     // per CTA: 1 + the last iteration whose reduction it published
  unsigned* rbcnt;     // per row block: arrivals of its K-split products (nks per iteration)
  int* status;
  int nb, npi, r0, k_pi, q, mmax;
  int kpad, nrb, nks, kc, nc, rpb;   // rpb: rows of its row block that a CTA reduces
  double* sig2;
  double* ritz;
};

// 16 consecutive FP32 columns of one TMEM accumulator, this warp's 32 lanes
// (rows); the caller waits with tcgen05.wait::ld before reading r.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ int tc_col_rows(const TcArgs& a, int c) {
  const int pcol = 2 * a.npi;
  if (c < pcol) return (c < a.nb) ? a.r0 + c + 1 : 0;
  return a.r0 + ((c - pcol) >> 1) + 1;
}

__device__ __forceinline__ void split_levels(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__device__ __forceinline__ void eig2_sym_tc(double s00, double s01, double s11, double& l0, double& l1, double& v00,
                                            double& v01, double& v10, double& v11) {
  const double tr = 0.5 * (s00 + s11), df = 0.5 * (s00 - s11);
  const double rad = sqrt(df * df + s01 * s01);
  l0 = tr + rad;
  l1 = tr - rad;
  if (rad == 0.0) { v00 = 1; v10 = 0; v01 = 0; v11 = 1; return; }
  const double th = 0.5 * atan2(2.0 * s01, s00 - s11);
  v00 = cos(th); v10 = sin(th); v01 = -v10; v11 = v00;
}

// Final values of the pairs whose last product was iteration `fin_it`, from
// the partial sums that every CTA wrote in that iteration's reduction
// (FP64 over the CTAs, spread over the CTAs); warp w0 the power-iteration
// estimates, warp w1 the Rayleigh-Ritz values of the k = 2 step.
__device__ __forceinline__ void tc_finals(const TcArgs& a, const float* s, int fin_it, int warp, int lane, int w0,
                                          int w1) {
  const int G = gridDim.x, blk = blockIdx.x;
  if (fin_it == a.k_pi && warp == w0) {
    for (int t = blk; t < a.nb; t += G) {
      const float* q0 = s + (size_t)((t >> 1) * kTcSlots + (t & 1)) * G;
      double v = 0.0;
      for (int g = lane; g < G; g += 32) v += (double)__ldcg(q0 + g);
      v = warp_sum(v);
      if (lane == 0) a.sig2[t] = v;
    }
  }
  if (fin_it == a.q && warp == w1) {
    for (int t = blk; t < a.nb; t += G) {
      const float* q0 = s + (size_t)((a.npi + t) * kTcSlots) * G;
      double v[kTcSlots];
#pragma unroll
      for (int e = 0; e < kTcSlots; ++e) {
        double x = 0.0;
        for (int g = lane; g < G; g += 32) x += (double)__ldcg(q0 + (size_t)e * G + g);
        v[e] = warp_sum(x);
      }
      if (lane == 0) {
        // S = X^T G X, H = (G X)^T (G X); G-orthonormal W = X V diag(a),
        // Ritz values = eig(diag(a) V^T H V diag(a))
        double l0, l1, v00, v01, v10, v11;
        eig2_sym_tc(v[0], v[1], v[2], l0, l1, v00, v01, v10, v11);
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

// Synchronisation.  No grid-wide barrier: a row block's K-split products and
// their reduction are separated by a counter of that row block alone (each of
// its nks CTAs adds one per iteration, release, and waits for nks (it + 1),
// acquire).  The reduction of CTA (rb, ks) publishes rows
// rb 128 + [ks rpb, (ks+1) rpb) of Y_{it+1} and its partial sums with a
// release store of flags[cta] = it + 1; the product of the next iteration
// waits (acquire) only for the flags of the CTAs whose rows form its K range,
// and the coefficient warps, which need every CTA's partial sums, wait for all
// flags while the product runs, so no CTA starts the reduction of iteration
// it + 1 before every CTA has finished that of iteration it.  With the
// products, Y and the partial sums double buffered by iteration parity, no
// buffer is then written while a slower CTA still reads it: a CTA writes only
// its own row block's rows of the product planes, and a CTA at iteration it + 2
// has waited for everyone's reduction of it + 1.
// SPL bounds the K splits the reduction sums (nks <= SPL); with SPL = 8 a
// round of the reduction issues the loads of four steps instead of two
// (six steps, all 96 pairs of a block in one round, measured slower: 427
// against 411 us per launch).
template <int NPASS, int SPL>
__global__ void __launch_bounds__(kTcThreads, 1) batch_tc_kernel(const TcArgs a,
                                                                 const __grid_constant__ UmmaOperand mG,
                                                                 const __grid_constant__ UmmaOperand mY) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s: [G level 0][G level 1][Y level 0][Y level 1] of one 64-wide K tile
  const uint32_t A_BYTES = UM * UK * 2;
  const uint32_t B_BYTES = (uint32_t)a.nc * UK * 2;
  const uint32_t S_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  __shared__ __align__(8) uint64_t full_bar[kTcStages];
  __shared__ __align__(8) uint64_t empty_bar[kTcStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int fail_s;
  __shared__ float4 coef[kTcMaxCols / 2];
  __shared__ int rb_ok_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, blk = blockIdx.x;
  const int rb = blk / a.nks, ks = blk - rb * a.nks;
  const int P = a.npi + a.nb;
  const int k0 = ks * a.kc, k1 = min(a.kpad, k0 + a.kc);
  const int ktiles = (k1 > k0) ? (k1 - k0) / UK : 0;
  const int niter = ktiles;   // one ring step per K tile; the NPASS level products share it
  static_assert(NPASS == 3, "the ring holds two levels of each operand");

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&done_bar, 1);
    fail_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {   // two accumulators of nc columns (<= 384): all 512 TMEM columns of the SM
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.nc >> 3) << 17) |
                         ((uint32_t)(UM >> 4) << 24);

  const int iters = max(a.k_pi, a.q);
  bool alive = true;
  for (int it = 0; it <= iters; ++it) {
    const bool pi_on = it <= a.k_pi, si_on = it <= a.q;
    const int pa0 = pi_on ? 0 : a.npi, pa1 = si_on ? P : a.npi;
    const int nact = pa1 - pa0;
    const int bold = (it + 1) & 1, bnew = it & 1;
    const float* Yold = a.Y + (size_t)bold * a.ybuf;
    float* Ynew = a.Y + (size_t)bnew * a.ybuf;
    const float* sold = a.sums + (size_t)bold * a.sbuf;
    float* snew = a.sums + (size_t)bnew * a.sbuf;
    float* part = a.part + (size_t)bnew * a.nks * a.pplane;

    // ---- product phase: Z(rows rb, all columns) over K range ks ----
    if (warp == 0 && niter > 0) {
      bool ok = true;
      if (it > 0) {
        // rows [k0, k1) of Y_it: the reductions of the previous iteration that
        // hold them; the warp's lanes poll those CTAs' flags at the same time
        // (one L2 round trip when they are set, not one per flag)
        // CTA (rb', ks') reduced rows rb' 128 + [ks' rpb, (ks'+1) rpb)
        const int rb_lo = k0 / UM, rb_hi = (k1 - 1) / UM;
        const int ncand = (rb_hi - rb_lo + 1) * a.nks;
        for (int e = lane; e < ncand; e += 32) {
          const int rbx = rb_lo + e / a.nks, ksx = e - (e / a.nks) * a.nks;
          const int lo = rbx * UM + ksx * a.rpb, hi = min(rbx * UM + UM, lo + a.rpb);
          if (lo < k1 && hi > k0 && ok) ok = wait_flag_ge(a.flags + rbx * a.nks + ksx, (unsigned)it, a.status);
        }
      }
      ok = __all_sync(0xffffffffu, ok);
      if (lane == 0 && ok) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");          // the other lanes' acquires, for lane 0
        asm volatile("fence.proxy.async.global;" ::: "memory");   // Y_it was written through the generic proxy
      }
      for (int li = 0; li < niter && ok && lane == 0; ++li) {
        const int g = it * niter + li;
        const int s = g % kTcStages;
        const uint32_t ph = (uint32_t)(g / kTcStages) & 1u;
        if (!mbar_wait(&empty_bar[s], ph ^ 1u)) { ok = false; break; }
        const int kx = k0 + li * UK;
        uint8_t* st = smem + (size_t)s * S_BYTES;
        mbar_expect_tx(&full_bar[s], S_BYTES);
        tma_load_2d(st, &mG.m[0], &full_bar[s], kx, rb * UM);
        tma_load_2d(st + A_BYTES, &mG.m[1], &full_bar[s], kx, rb * UM);
        tma_load_2d(st + 2 * A_BYTES, &mY.m[0], &full_bar[s], kx, bold * a.ycols);
        tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mY.m[1], &full_bar[s], kx, bold * a.ycols);
      }
      if (lane == 0 && !ok) atomicExch(&fail_s, 1);
    } else if (warp == 1) {
      if (lane == 0 && niter > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int li = 0; li < niter; ++li) {
          const int g = it * niter + li;
          const int s = g % kTcStages;
          const uint32_t ph = (uint32_t)(g / kTcStages) & 1u;
          if (!mbar_wait(&full_bar[s], ph)) { atomicExch(&fail_s, 1); break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + (size_t)s * S_BYTES);
          // level products G0 Y0 (leading accumulator), G0 Y1 and G1 Y0 (corrections)
  #pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t a0 = st + (pass == 2 ? A_BYTES : 0u);
            const uint32_t b0 = st + 2 * A_BYTES + (pass == 1 ? B_BYTES : 0u);
  #pragma unroll
            for (int kk = 0; kk < UK / 16; ++kk) {
              const int aidx = (pass == 0) ? 0 : 1;
              const bool first = (li == 0) && (kk == 0) && (pass <= 1);
              const uint32_t dst = tmem + (uint32_t)(aidx * a.nc);
              const uint64_t da = smem_desc(a0 + kk * 32), db = smem_desc(b0 + kk * 32);
              const uint32_t acc = first ? 0u : 1u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                  "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty_bar[s]))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done_bar))
                     : "memory");
      }
      __syncwarp();
      // the row block's K-split products of this iteration are all written once
      // the epilogue warps (4-7) pass barrier 2: this CTA arrives (release) and
      // waits (acquire, bounded) for the row block's other CTAs; no other row
      // block takes part
      asm volatile("bar.sync 2, 160;" ::: "memory");
      if (lane == 0) {
        if (fail_s) set_status(a.status, AS_ETIMEOUT);
        red_release_add_u32(a.rbcnt + rb, 1u);
        rb_ok_s = wait_flag_ge(a.rbcnt + rb, (unsigned)(it + 1) * (unsigned)a.nks, a.status) ? 1 : 0;
      }
    } else if (warp >= 2) {
      if (warp >= 4) {
        // epilogue: warps 4-7 (TMEM lane quarters 0-3) move the 128 x nc block,
        // both accumulators summed, to part[ks]; the MMAs are waited for even
        // after a failure, so none is in flight when the TMEM is freed
        const int wq = warp - 4;
        bool have = niter > 0 && mbar_wait(&done_bar, (uint32_t)it & 1u);
        if (niter > 0 && !have) atomicExch(&fail_s, 1);
        if (fail_s) have = false;
        have = __all_sync(0xffffffffu, have);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = rb * UM + wq * 32 + lane;
        float* o = part + (size_t)ks * a.pplane + (size_t)row * a.nc;
        const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);
        // 32 columns of both accumulators per wait (nc is a multiple of 16)
        for (int c0 = 0; c0 < a.nc && niter > 0; c0 += 32) {
          const bool two = c0 + 16 < a.nc;   // warp-uniform
          uint32_t r[4][16];
          if (have) {
            tmem_ld16(trow + (uint32_t)c0, r[0]);
            tmem_ld16(trow + (uint32_t)(c0 + a.nc), r[1]);
            if (two) {
              tmem_ld16(trow + (uint32_t)(c0 + 16), r[2]);
              tmem_ld16(trow + (uint32_t)(c0 + 16 + a.nc), r[3]);
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
              v[j] = have ? __uint_as_float(r[2 * h][j]) + __uint_as_float(r[2 * h + 1][j]) : 0.f;
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              __stcg(reinterpret_cast<float4*>(o + c0 + 16 * h + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync 2, 160;" ::: "memory");   // with warp 1: the product is written
      }
      // coefficients C_it of the active pairs from every CTA's partial sums of Y_it
      constexpr int kCT = kTcThreads - 64;
      const int ct = tid - 64;
      if (it == 0) {
        for (int p = ct; p < P; p += kCT) coef[p] = make_float4(1.f, 0.f, 0.f, 1.f);
      } else {
        bool ok = true;
        for (int c = ct; c < G && ok; c += kCT) ok = wait_flag_ge(a.flags + c, (unsigned)it, a.status);
        if (!ok) atomicExch(&fail_s, 1);
        __syncwarp();
        asm volatile("bar.sync 1, %0;" ::"r"(kCT) : "memory");
        // pairs whose last product was the previous iteration: their final values
        tc_finals(a, sold, it - 1, warp, lane, 2, 3);
        for (int pbase = pa0 + 4 * (warp - 2); pbase < pa1; pbase += 4 * (kCT / 32)) {
          float sv[4][3];
#pragma unroll
          for (int j = 0; j < 4; ++j) sv[j][0] = sv[j][1] = sv[j][2] = 0.f;
          for (int g0 = 0; g0 < G; g0 += 128) {
            float buf[4][4][3];
#pragma unroll
            for (int gg = 0; gg < 4; ++gg) {
              const int g = g0 + 32 * gg + lane;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int p = pbase + j;
                const bool on = p < pa1 && g < G;
                const float* q0 = sold + (size_t)(p * kTcSlots) * G + g;
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
            coef[p] = make_float4(c00, c10, c01, c11);
          }
        }
      }
    }
    // a block barrier is executed by converged warps only: warps 0 and 1 may
    // still be split (lane 0 alone ran the producer or the row-block wait)
    __syncwarp();
    __syncthreads();   // coefficients, the row block's products and rb_ok_s
    if (!rb_ok_s) { alive = false; break; }

    // ---- reduction phase: rows [rw0, rw1) of row block rb of Y_{it+1} = Z C_it ----
    // A group of lpp lanes (a half warp for up to 16 rows, else a warp) takes
    // one column pair, one row per lane: the K-split planes of its row are
    // summed in the order k = 0, 1, ..., the row of Y_{it+1} is written in FP32
    // and BF16 levels (consecutive lanes, consecutive rows: coalesced), and the
    // pair's partial sums are reduced across the group.  The loads of two
    // steps are issued before either step's arithmetic.
    const int rw0 = rb * UM + ks * a.rpb, rw1 = min(rb * UM + UM, rw0 + a.rpb);
    const int R = max(0, rw1 - rw0);
    const int lpp = (R <= 16) ? 16 : 32;
    const int sub = (lpp == 16) ? (lane >> 4) : 0, rl = lane & (lpp - 1);
    const int pstep = kTcThreads / lpp;   // pairs per step (all warps)
    const int row = rw0 + rl;
    const bool row_on = rl < R;
    const bool in_y = row < a.ldy;        // rows past the FP32 columns are zero (>= m_t)
    constexpr int HS = 32 / SPL;          // steps whose loads go out together
    for (int pb0 = 0; pb0 < nact; pb0 += HS * pstep) {
      float2 zz[HS][SPL];
#pragma unroll
      for (int h = 0; h < HS; ++h) {
        const int pl = pb0 + h * pstep + warp * (32 / lpp) + sub;
        const bool on = pl < nact && row_on;
        const float* pp = part + (size_t)row * a.nc + 2 * (pa0 + pl);
#pragma unroll
        for (int k = 0; k < SPL; ++k)
          zz[h][k] = (on && k < a.nks) ? __ldcg(reinterpret_cast<const float2*>(pp + (size_t)k * a.pplane))
                                       : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int h = 0; h < HS; ++h) {
        const int pl = pb0 + h * pstep + warp * (32 / lpp) + sub;
        const bool pon = pl < nact;
        const bool on = pon && row_on;
        const int p = pa0 + (pon ? pl : 0);
        float za = 0.f, zb = 0.f;
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
          za += zz[h][k].x;
          zb += zz[h][k].y;
        }
        const bool si = p >= a.npi;
        const bool fin = si ? (it == a.q) : (it == a.k_pi);
        const float4 cf = coef[p];
        const int ca = 2 * p, cb = 2 * p + 1;
        const int ma = tc_col_rows(a, ca), mb = tc_col_rows(a, cb);
        const float y0 = (on && row < ma) ? fmaf(cf.x, za, cf.y * zb) : 0.f;
        const float y1 = (on && row < mb) ? fmaf(cf.z, za, cf.w * zb) : 0.f;
        float ps[kTcSlots] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (on) {
          if (in_y) {
            Ynew[(size_t)ca * a.ldy + row] = y0;
            Ynew[(size_t)cb * a.ldy + row] = y1;
          }
          __nv_bfloat16 l0, l1, l2;
          split_levels(y0, l0, l1, l2);
          __nv_bfloat16* ya = a.Yb + (size_t)bnew * a.ybbuf + (size_t)ca * a.ldyb + row;
          ya[0] = l0;
          ya[a.yblevel] = l1;
          ya[2 * a.yblevel] = l2;
          split_levels(y1, l0, l1, l2);
          __nv_bfloat16* yb = ya + a.ldyb;
          yb[0] = l0;
          yb[a.yblevel] = l1;
          yb[2 * a.yblevel] = l2;
          if (!fin) {
            ps[0] = y0 * y0;
            if (si) {
              ps[1] = y0 * y1;
              ps[2] = y1 * y1;
            } else {
              ps[1] = y1 * y1;
            }
          } else {
            // x = Y_it C_it (the normalised iterate), y = G x
            const float ya0 = in_y ? __ldcg(Yold + (size_t)ca * a.ldy + row) : 0.f;
            const float yb0 = in_y ? __ldcg(Yold + (size_t)cb * a.ldy + row) : 0.f;
            const float x0 = fmaf(cf.x, ya0, cf.y * yb0), x1 = fmaf(cf.z, ya0, cf.w * yb0);
            if (!si) {
              ps[0] = x0 * y0;
              ps[1] = x1 * y1;
            } else {
              ps[0] = x0 * y0;
              ps[1] = 0.5f * fmaf(x0, y1, x1 * y0);
              ps[2] = x1 * y1;
              ps[3] = y0 * y0;
              ps[4] = y0 * y1;
              ps[5] = y1 * y1;
              if (row < a.ldx) {
                a.X[(size_t)ca * a.ldx + row] = x0;
                a.X[(size_t)cb * a.ldx + row] = x1;
              }
            }
          }
        }
        // the pair's partial sums over its rows (every lane takes part)
#pragma unroll
        for (int e = 0; e < kTcSlots; ++e)
          for (int o = lpp >> 1; o > 0; o >>= 1) ps[e] += __shfl_xor_sync(0xffffffffu, ps[e], o);
        if (pon && rl == 0) {
#pragma unroll
          for (int e = 0; e < kTcSlots; ++e) snew[(size_t)(p * kTcSlots + e) * G + blk] = ps[e];
        }
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");   // the BF16 levels feed other CTAs' TMA loads
    __syncwarp();
    __syncthreads();
    if (tid == 0) st_release_u32(a.flags + blk, (unsigned)(it + 1));
  }
  // the pairs whose last product was the final iteration
  if (alive) {
    __shared__ int ok_s;
    if (tid == 0) ok_s = 1;
    __syncwarp();
    __syncthreads();
    for (int c = tid; c < G; c += kTcThreads)
      if (!wait_flag_ge(a.flags + c, (unsigned)(iters + 1), a.status)) ok_s = 0;
    __syncwarp();
    __syncthreads();
    if (ok_s) tc_finals(a, a.sums + (size_t)(iters & 1) * a.sbuf, iters, warp, lane, 0, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  __syncthreads();
  if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// x^(0) and Pi of every row (FP32, buffer 1) as the FP32 form writes them,
// then their BF16 levels for rows [0, kpad) of columns [0, ncols).
__global__ void tc_split_start_kernel(const float* Y, int ldy, int mmax, int ncols, int kpad, __nv_bfloat16* Yb,
                                      long long yblevel, int ldyb) {
  const int c = blockIdx.x;
  if (c >= ncols) return;
  for (int r = threadIdx.x; r < kpad; r += blockDim.x) {
    const float v = (r < mmax) ? Y[(size_t)c * ldy + r] : 0.f;
    __nv_bfloat16 l0, l1, l2;
    split_levels(v, l0, l1, l2);
    __nv_bfloat16* o = Yb + (size_t)c * ldyb + r;
    o[0] = l0;
    o[yblevel] = l1;
    o[2 * yblevel] = l2;
  }
}

// BF16 levels of rows and columns [valid, m) of the leading m x m block of G,
// and the same entries of the FP32 mirror Gf (ld n2) when it is given.
__global__ void tc_mirror_kernel(const double* G, int n2, int valid, int m, __nv_bfloat16* Gb, long long level,
                                 int ldg, float* Gf) {
  const int p = blockIdx.x;
  if (p >= m) return;
  const int q0 = (p < valid) ? valid : 0;
  for (int q = q0 + threadIdx.x; q < m; q += blockDim.x) {
    const double x = G[(size_t)p * n2 + q];
    __nv_bfloat16 l0, l1, l2;
    g_levels(x, l0, l1, l2);
    __nv_bfloat16* o = Gb + (size_t)p * ldg + q;
    o[0] = l0;
    o[level] = l1;
    o[2 * level] = l2;
    if (Gf) Gf[(size_t)p * n2 + q] = (float)x;
  }
}

struct TcDevice {
  int sms = 0;
  size_t attr[2] = {0, 0};
};
TcDevice g_tcdev[64];
std::mutex g_tcdev_mu;

}  // namespace

as_status launch_tc_mirror(cudaStream_t s, const double* G, int n2, int valid, int m, const TcBatchBuffers& tb,
                           float* Gf) {
  if (m <= 0 || valid >= m) return AS_OK;
  tc_mirror_kernel<<<m, 256, 0, s>>>(G, n2, std::max(valid, 0), m, tb.Gb, tb.glevel, tb.ldg, Gf);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

size_t batch_tc_part_floats(int n2, int ycols) {
  const size_t kpad = (size_t)(n2 + 127) / 128 * 128;
  // two buffers of nks <= 16 planes (checked at launch), then 256 CTA flags
  // and 256 row-block counters
  return (size_t)2 * 16 * kpad * (size_t)std::min(ycols, kTcMaxCols) + 512;
}

as_status launch_batch_tc_prefill(cudaStream_t s, int n2, int r0, int nb, Key key, uint64_t i0,
                                  const PersistBuffers& pb, const TcBatchBuffers& tb, bool* done) {
  *done = false;
  if (nb <= 0) return AS_OK;
  const int mmax = r0 + nb;
  const int npi = (nb + 1) / 2, P = npi + nb;
  const int kpad = (mmax + 127) / 128 * 128;
  const int ncols = 2 * P;
  const int nc = (ncols + 15) / 16 * 16;
  if (kpad < 256 || nc > kTcMaxCols || nc > (int)pb.ycols) return AS_OK;
  launch_persist_fill(s, pb, mmax, nb, npi, r0, key, i0);
  tc_split_start_kernel<<<ncols, 256, 0, s>>>(pb.Y + pb.ybuf, pb.ldy, mmax, ncols, kpad,
                                              tb.Yb + (size_t)pb.ycols * tb.ldyb, tb.yblevel, tb.ldyb);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  unsigned* flags = reinterpret_cast<unsigned*>(tb.part + batch_tc_part_floats(n2, (int)pb.ycols) - 512);
  AS_CUDA_TRY(cudaMemsetAsync(flags, 0, 512 * sizeof(unsigned), s));
  *done = true;
  return AS_OK;
}

as_status launch_batch_tc(cudaStream_t s, int n2, int r0, int nb, int k_pi, int q, Key key, uint64_t i0,
                          const PersistBuffers& pb, const TcBatchBuffers& tb, int npass, int* status, Prof* prof,
                          bool* used, bool prefilled) {
  *used = false;
  if (nb <= 0) return AS_OK;
  const int mmax = r0 + nb;
  const int npi = (nb + 1) / 2, P = npi + nb;
  const int kpad = (mmax + 127) / 128 * 128;
  const int ncols = 2 * P;
  const int nc = (ncols + 15) / 16 * 16;
  if (kpad < 256 || nc > kTcMaxCols || nc > (int)pb.ycols || npass != 3) return AS_OK;
  int dev = 0;
  AS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return AS_OK;
  std::unique_lock<std::mutex> lk(g_tcdev_mu);
  TcDevice& td = g_tcdev[dev];
  if (td.sms == 0) AS_CUDA_TRY(cudaDeviceGetAttribute(&td.sms, cudaDevAttrMultiProcessorCount, dev));
  // K range per CTA: by default as short as the co-resident grid (one CTA per
  // SM) allows; the autotuner may take two or four times fewer K splits
  // (fewer partial planes to reduce, more MMA work per CTA)
  const int nrb = kpad / 128;
  const long long need = ((long long)kpad * kpad + 128LL * td.sms - 1) / (128LL * td.sms);
  const int kc0 = (int)std::max<long long>(64, (need + 63) / 64 * 64);
  const int nks0 = (kpad + kc0 - 1) / kc0;
  const size_t smem = 1024 + (size_t)kTcStages * 2 * (UM * UK * 2 + (size_t)nc * UK * 2);
  const void* fns[2] = {(const void*)batch_tc_kernel<3, 8>, (const void*)batch_tc_kernel<3, 16>};
  int per = 1 << 30;
  for (int v = 0; v < 2; ++v) {
    if (smem > td.attr[v]) {
      AS_CUDA_TRY(cudaFuncSetAttribute(fns[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      td.attr[v] = smem;
    }
    int pv = 0;
    AS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pv, fns[v], kTcThreads, smem));
    per = std::min(per, pv);
  }
  const int sms = td.sms;
  lk.unlock();
  // the split shape of a candidate K-split count: (kc, nks) with kc a multiple
  // of 64, or nks = 0 when the shape does not fit
  auto shape = [&](int want, int* kc_out) -> int {
    if (want < 1) return 0;
    int kc = (kpad + want - 1) / want;
    kc = (kc + 63) / 64 * 64;
    const int nks = (kpad + kc - 1) / kc;
    const int rpb = (UM + nks - 1) / nks;
    if (nks > kTcMaxSplits || rpb > kTcMaxRpc || nrb * nks > sms || per < 1 || (long long)per * sms < nrb * nks)
      return 0;
    *kc_out = kc;
    return nks;
  };
  int choices[3], nch = 0;
  for (int f = 1; f <= 4; f *= 2) {
    int kc = 0;
    const int nks = shape((nks0 + f - 1) / f, &kc);
    bool dup = false;
    for (int c = 0; c < nch; ++c) dup = dup || choices[c] == nks;
    if (nks > 0 && !dup) choices[nch++] = nks;
  }
  if (nch == 0) return AS_OK;
  // the BF16 levels of the batch vectors: two buffers of ycols columns per level
  UmmaOperand mY{};
  for (int l = 0; l < 3; ++l) {
    as_status st = umma_make_map(&mY.m[l], tb.Yb + (size_t)l * tb.yblevel, 2 * (int)pb.ycols, tb.ldyb, tb.ldyb, nc);
    if (st != AS_OK) return st;
  }
  unsigned* flags = reinterpret_cast<unsigned*>(tb.part + batch_tc_part_floats(n2, (int)pb.ycols) - 512);
  // one launch of the block with nks K splits: starting vectors (unless the
  // caller filled them already, launch_batch_tc_prefill), then the kernel;
  // every tuning run refills them, since the kernel overwrites them
  bool tuning = false;
  auto run = [&](int want) -> as_status {
    int kc = 0;
    const int nks = shape(want, &kc);
    if (nks == 0) return AS_ENOTSUP;
    const int ncta = nrb * nks, rpb = (UM + nks - 1) / nks;
    if (tuning || !prefilled) {
      if (prof) prof->begin(PK_BATCH_ORTH, s);
      launch_persist_fill(s, pb, mmax, nb, npi, r0, key, i0);
      tc_split_start_kernel<<<ncols, 256, 0, s>>>(pb.Y + pb.ybuf, pb.ldy, mmax, ncols, kpad,
                                                  tb.Yb + (size_t)pb.ycols * tb.ldyb, tb.yblevel, tb.ldyb);
      count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
      if (prof) prof->end(PK_BATCH_ORTH, s, 0.0, 12.0 * mmax * (double)nb);
      AS_CUDA_TRY(cudaMemsetAsync(flags, 0, 512 * sizeof(unsigned), s));   // CTA flags and row-block counters
    }
    TcArgs a{};
    a.Y = pb.Y; a.ybuf = pb.ybuf; a.ldy = pb.ldy;
    a.Yb = tb.Yb; a.yblevel = tb.yblevel; a.ybbuf = (long long)pb.ycols * tb.ldyb; a.ldyb = tb.ldyb;
    a.ycols = (int)pb.ycols;
    a.X = pb.X; a.ldx = n2;
    a.part = tb.part; a.pplane = (long long)kpad * nc;
    a.sums = pb.part; a.sbuf = (long long)kTcSlots * P * ncta;
    a.flags = flags; a.rbcnt = flags + 256; a.status = status;
    a.nb = nb; a.npi = npi; a.r0 = r0; a.k_pi = k_pi; a.q = q; a.mmax = mmax;
    a.kpad = kpad; a.nrb = nrb; a.nks = nks; a.kc = kc; a.nc = nc; a.rpb = rpb;
    a.sig2 = pb.sig2; a.ritz = pb.ritz;
    void* args[] = {&a, (void*)&tb.mG, &mY};
    if (prof) prof->begin(PK_BATCH_TC, s);
    AS_CUDA_TRY(cudaLaunchCooperativeKernel(fns[nks <= 8 ? 0 : 1], dim3(ncta), dim3(kTcThreads), args, smem, s));
    count_launches(1);
    if (prof) {
      double m2 = 0.0;
      for (int t = 0; t < nb; ++t) {
        const double m = (double)(r0 + t + 1);
        m2 += m * m;
      }
      const double prods = (double)(k_pi + 1) + 2.0 * (double)(q + 1);
      // the algorithmic work of the block is recorded when its decisions are
      // taken (add_work); here the work issued for every row of the block, and
      // the algorithmic DRAM bytes: the two BF16 levels of G read once (Y and
      // the partial planes stay in L2)
      prof->end(PK_BATCH_TC, s, 0.0, 4.0 * (double)kpad * kpad, 2.0 * m2 * prods);
    }
    return AS_OK;
  };
  as_status st = AS_OK;
  bool ran = false;
  tuning = true;
  const int nks = tune_pick(s, "batch_tc_nks", kpad, choices, nch, run, &st, &ran);
  tuning = false;
  if (st != AS_OK) return st;
  if (!ran) {
    st = run(nks);
    if (st != AS_OK) return st;
  }
  *used = true;
  return AS_OK;
}

}  // namespace as

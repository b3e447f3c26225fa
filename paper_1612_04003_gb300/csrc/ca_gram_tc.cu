// ca_gram_tc.cu -- the fused gather + Gram + projection pass on the sm_103a
// tensor cores (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// One outer step of CA-BCD (Alg. 2) / CA-BDCD (Alg. 4) needs, from the s*b
// sampled rows Y of A (primal A = X; dual A = X^T), the Gram matrix Y Y^T and
// the projection Y v (primal v = y - z, dual v = w), both in one pass over Y
// ("compute the Gram matrix" of Alg. 2 / 4).  This kernel makes that pass:
//
//  * grid = P CTAs, one per SM; CTA c owns a contiguous range of 32-column
//    K-atoms and produces split-K partials (the single-GPU counterpart of the
//    paper's all-reduce of the Gram matrix, Sec. 4);
//  * A is row-major, or (in the solves) stored as 32-column panels
//    [K/32][N][32]: a stage's sampled rows then lie in one N x 128-byte block
//    instead of N rows a full row length apart, which lets the gather run
//    at a higher fraction of HBM bandwidth (fewer pages and DRAM rows per stage);
//  * warps 0-7 gather the sampled rows with 16-byte cp.async straight into
//    the 128-byte-swizzled K-major layout that tcgen05.mma reads (8-row atoms
//    of 1024 bytes, 16-byte chunk c of row r stored at chunk c ^ (r % 8)),
//    NS stages deep; the same warps form the projection from the staged tile
//    on CUDA cores (v split into two FP32 halves, FP32 products, compensated
//    FP32 sums);
//  * warp 8 allocates tensor memory and one thread issues the MMAs
//    (M = 128; N = the padded s*b) accumulating Y Y^T in TMEM;
//  * after the K loop warps 0-7 read TMEM (tcgen05.ld) and store the FP32
//    partial tile(s) that cover the lower triangle.
// With three_pass the FP32 inputs are split into a TF32 head and a TF32 tail
// (x = hi + lo) and hi*hi + hi*lo + lo*hi are accumulated (3xTF32); the
// loaders write hi and lo into a separate 2-slot operand ring, so the load
// ring never waits on the tensor cores.
// With a fused update (s*b <= 128) each stage also brings in the previous
// outer step's rows: the loader warps apply that step's deferred update
// (v -= cU Yprev^T Delta: FP32 products of the FP32 rows with the (hi, lo)
// FP32 split of Delta, summed in FP32, the result applied in double-float to
// the FP32-pair copy of v) to the stage's 32 columns, write it back, and
// project the current rows on the updated values: the update pass and the
// next Gram pass share one launch and one sweep over the K range.
// Every wait is bounded (CA_WAIT_LIMIT_NS) and raises CA_DEV_ERR_TIMEOUT.
#include <atomic>

#include "ca_kernels.cuh"
#include "ca_tc.cuh"

namespace {

constexpr int kLoaderWarps = 8;                      // 2 per SM sub-partition
constexpr int kLoaderThreads = 32 * kLoaderWarps;    // loaders / projection / epilogue
constexpr int kMmaWarp = kLoaderWarps;               // TMEM allocation and MMA issue
constexpr int kThreads = kLoaderThreads + 32;

template <int SBP, bool THREE, bool UPD = false, bool BF = false, bool F16 = false>
struct TcCfg {
  static constexpr int kTileBytes = SBP * 128;                  // SBP rows x 32 fp32
  // operand tiles of the split modes: 3xTF32 rows of 32 fp32 (128-byte
  // swizzle), BF16x3 rows of 32 bf16 (64 bytes, 64-byte swizzle)
  static constexpr int kOpRow = BF ? 64 : 128;
  static constexpr int kOpTile = SBP * kOpRow;
  // cp.async slot: [current rows | previous step's rows (fused update)]
  static constexpr int kRawBytes = kTileBytes * (UPD ? 2 : 1);
  static constexpr int kPrevOff = kTileBytes;
  // 3xTF32: the loaders write the (head, tail) tiles into a separate ring of
  // kMS slots that the MMA reads, so a load slot is free again as soon as its
  // own thread has consumed it (no wait on the MMA before a refill).  Plain
  // TF32: the MMA reads the load slot itself.
  // (scaled FP16: one tile, x s_r rounded to FP16, one product)
  static constexpr int kMmaSlotBytes = THREE ? (F16 ? 1 : 2) * kOpTile : 0;
  static constexpr int kBudget = 200 * 1024;                    // both rings
  static constexpr int kMS =
      THREE ? ((kBudget - 2 * kMmaSlotBytes) / kRawBytes >= 4 ? 2 : 1) : 0;
  static constexpr int kNSfit = (kBudget - kMS * kMmaSlotBytes) / kRawBytes;
  static constexpr int kNS = kNSfit < 16 ? kNSfit : 16;         // load-ring depth
  static constexpr int kMmaRing = kMS * kMmaSlotBytes;
  // one FP32 accumulator per 128-row tile; the split modes add their three
  // products (hi hi^T, hi lo^T, lo hi^T) into it (a second accumulator for
  // hi lo^T, transposed through shared memory in the epilogue, measured
  // 1.3 us slower per launch)
  // (SBP 256: rows 128..255 against up to 256 columns at column 128; the
  // allocation is a power of two)
  static constexpr int kTmemCols = (SBP == 256) ? 512 : 128;
  // the M = 128 MMA reads 128 rows of its A tile; with SBP < 128 the rows past
  // the tile are whatever follows in shared memory (their accumulator rows
  // are never stored).  The MMA ring is followed by the load ring; the last
  // load slot (plain TF32) needs that much slack behind it.
  static constexpr int kSlack = (!THREE && kRawBytes < 16384) ? 16384 - kRawBytes : 0;
  static constexpr int kRPT = SBP / 32;                         // rows per loader thread
  // projection-vector ring: 2*NS slots of 32 (hi, lo) pairs, so that a slot is
  // rewritten only after every loader passed the barrier of a later stage
  static constexpr int kVRing = 2 * kNS * 256;
  // fused update: per-warp column sums, double-buffered by stage parity
  static constexpr int kUpdBytes = UPD ? 2 * kLoaderWarps * 32 * 4 : 0;
  static constexpr int kZeroBytes = kMmaRing + kNS * kRawBytes + kVRing + kUpdBytes + kSlack;
  static constexpr int kSmem = kZeroBytes + 1024 + 512;
  static_assert(THREE || kNS >= 4, "plain TF32 refills one stage late: needs >= 4 slots");
  static_assert(kNS >= 2, "load ring too shallow");
  static_assert(kSmem <= 232448, "shared memory");
};

// One unit of work of a CTA: 32-column atoms [a0, a1) of one problem's sampled
// rows, accumulated into one split-K partial slot.
struct GramUnitArgs {
  const float* A;
  long long lda, N, K;
  const int* idx;
  int sb;
  const float2* v2;
  long long a0, a1;
  float* part;     // SBP x SBP partial tile of this unit (stored transposed)
  double* ppart;   // SBP projection partials of this unit
  GramUpdate u;
};

template <int SBP, bool THREE, bool UPD, bool PANEL, bool BF, bool F16, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const float* __restrict__ A, long long lda, long long N, long long K,
          const int* __restrict__ idx, int sb, const float2* __restrict__ v2, long long natoms,
          float* __restrict__ part, double* __restrict__ ppart, unsigned* __restrict__ err,
          GramUpdate u, GramBatchArgs bt) {
  using C = TcCfg<SBP, THREE, UPD, BF, F16>;
  static_assert(!F16 || (THREE && BF), "scaled FP16 uses the 16-bit operand ring");
  constexpr int NS = C::kNS, MS = C::kMS, RPT = C::kRPT;
  extern __shared__ unsigned char smem_raw[];
  // scaled FP16: 1 / multiplier of each tile row (exact powers of two)
  __shared__ float s_rinv[F16 ? SBP : 1];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* mring = smem;                    // MS x [head tile | tail tile] (3xTF32)
  unsigned char* raw = smem + C::kMmaRing;        // NS x [current rows | previous rows]
  unsigned char* vring = raw + NS * C::kRawBytes;  // 2*NS x 256 B
  float* ured = reinterpret_cast<float*>(vring + C::kVRing);  // [2][kLoaderWarps][32]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kZeroBytes);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;   // MMA -> epilogue, one phase per unit
  uint64_t* epi = done + 1;      // epilogue -> MMA (accumulator read), one phase per unit
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(epi + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x, P = gridDim.x;
  // the prologue below reads A, the sampled indices, v2 and the row scales:
  // before the preceding grid has finished only when it writes none of them
  if (!(BATCH ? bt.early : u.early)) pdl_wait();
  // this CTA's units: one (its even share of the atoms) or, in a shared
  // launch over several problems, the units the host's plan gave it
  const int nunits = BATCH ? bt.unit_begin[c + 1] - bt.unit_begin[c] : 1;
  auto unit = [&](int j) -> GramUnitArgs {
    if constexpr (BATCH) {
      const GramUnit gu = bt.units[bt.unit_begin[c] + j];
      const GramInst& gi = bt.insts[gu.inst];
      return GramUnitArgs{gi.A, gi.lda, gi.N, gi.K, gi.idx, gi.sb, gi.v2, gu.a0, gu.a1, gi.part + (long long)gu.slot * SBP * SBP,
                          gi.ppart + (long long)gu.slot * SBP, gi.u};
    } else {
      return GramUnitArgs{A, lda, N, K, idx, sb, v2, natoms * c / P, natoms * (c + 1) / P,
                          part + (long long)c * SBP * SBP, ppart + (long long)c * SBP, u};
    }
  };

  // Shared memory is not cleared: rows >= sb of a tile (never loaded) only
  // reach accumulator rows / columns >= sb and projection entries >= sb,
  // which are never stored or never read; the K tail past the last column is
  // zero-filled by the copies (row-major) or zero in the panels.
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {  // (3xTF32 uses the first MS pairs)
      mbar_init(&full[s], kLoaderWarps);  // one arrival per loader warp
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_init(epi, kLoaderWarps);
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp < kLoaderWarps) {
    // ---------------- loaders / projection / epilogue ----------------
    // Thread (g, l) copies, reads and converts 16-byte chunk l of rows
    // g + 32 i: a load slot holds only data its own thread consumes, so the
    // thread may refill it right after use.
    const int g = tid >> 3, l = tid & 7;
    uint32_t dsto[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = g + 32 * i;
      dsto[i] = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((l ^ (r & 7)) << 4));
    }
    const uint32_t raw0 = smem_u32(raw);
    const uint32_t vring0 = smem_u32(vring);
    bool ok = true;
    // one lane waits on the barrier, the warp follows; once a wait has timed
    // out no further waits are made (the per-stage slot wait polls on every
    // lane instead, which measured cheaper than the convergence)
    auto warp_wait = [&](uint64_t* bar, uint32_t parity, bool ok_in) -> bool {
      bool r = ok_in;
      if (lane == 0 && r) r = mbar_wait_bounded(bar, parity, err);
      r = __shfl_sync(0xffffffffu, r ? 1 : 0, 0) != 0;
      __syncwarp();
      return r;
    };
    // stages in flight ahead of the one being processed: 3xTF32 refills a
    // slot right after consuming it; plain TF32 refills the slot of the
    // previous stage once its MMA has completed
    constexpr int PRE = THREE ? NS : NS - 1;
    uint32_t g0 = 0;  // stages of the earlier units (ring slots and barrier phases run on)
    for (int j = 0; j < nunits; ++j) {
      const GramUnitArgs U = unit(j);
      const int T = (int)(U.a1 - U.a0);
      long long rowoff[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = g + 32 * i;
        const long long gi = (r < U.sb) ? (long long)U.idx[r] : -1;
        const bool in_range = gi >= 0 && gi < U.N;
        if (r < U.sb && !in_range) ca_flag(err, CA_DEV_ERR_ARG);  // skipped, never read
        rowoff[i] = in_range ? gi * (PANEL ? 32 : U.lda) : -1;
      }
      // scaled FP16: the multiplier of each of this thread's rows (a power of
      // two that brings the row's largest magnitude into [2^14, 2^15))
      float rsc[F16 ? RPT : 1];
      if constexpr (F16) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int r = g + 32 * i;
          rsc[i] = rowoff[i] >= 0 ? __ldg(U.u.rscale + U.idx[r]) : 1.f;
          if (l == 0) s_rinv[r] = 1.f / rsc[i];
        }
      }
      // fused update: this thread's rows of the previous outer step (their
      // Delta is read once the preceding grid has finished, below)
      const float2 u_cU2 = split_f64(U.u.cU);
      long long prevoff[UPD ? RPT : 1];
      float dph[UPD ? RPT : 1], dpl[UPD ? RPT : 1];
      if constexpr (UPD) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int r = g + 32 * i;
          const long long gi = (r < U.u.sb) ? (long long)U.u.idx[r] : -1;
          const bool in_range = gi >= 0 && gi < U.N;
          if (r < U.u.sb && !in_range) ca_flag(err, CA_DEV_ERR_ARG);
          prevoff[i] = in_range ? gi * (PANEL ? 32 : U.lda) : -1;
        }
      }
      auto issue = [&](int t, int slot) {
        // row-major: row gi, columns k .. k+3 at A + gi lda + k (the K tail is
        // zero-filled); panels: 32-column panel a of N rows x 128 B at
        // A + a N 32, zero-padded past K
        const long long k = (U.a0 + t) * 32 + 4 * l;
        uint32_t bytes = 16u;
        long long col = PANEL ? (U.a0 + t) * U.N * 32 + 4 * l : k;
        if constexpr (!PANEL) {
          const long long rem = U.K - k;
          bytes = rem >= 4 ? 16u : (rem > 0 ? (uint32_t)rem * 4u : 0u);
          if (!bytes) col = 0;
        }
        const uint32_t dst = raw0 + (uint32_t)(slot * C::kRawBytes);
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (rowoff[i] >= 0) cp_async_16_zfill(dst + dsto[i], U.A + rowoff[i] + col, bytes);
        if constexpr (UPD) {
#pragma unroll
          for (int i = 0; i < RPT; ++i)
            if (prevoff[i] >= 0)
              cp_async_16_zfill(dst + C::kPrevOff + dsto[i], U.A + prevoff[i] + col, bytes);
        }
        if (tid < 16)  // the stage's 32 (hi, lo) pairs of v (zero-padded to a multiple of 32)
          cp_async_16_zfill(vring0 + (uint32_t)(((g0 + t) % (2 * NS)) * 256 + tid * 16),
                            U.v2 + (U.a0 + t) * 32 + 2 * tid, 16u);
      };
      // projection accumulators: FP32 partial sums over 8 stages, folded into
      // a compensated (hi, lo) FP32 pair
      float pacc[RPT], phi[RPT], plo[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        pacc[i] = 0.f;
        phi[i] = 0.f;
        plo[i] = 0.f;
      }
      for (int t = 0; t < PRE; ++t) {
        if (t < T) issue(t, (int)((g0 + t) % NS));
        cp_async_commit();
      }
      if (j == 0) {
        // Everything above reads only X, the sampled indices, v2 and the row
        // scales; with early the preceding grid (the previous outer step's
        // solve) writes none of them.  Delta and the partial buffers wait for it.
        pdl_wait();
        pdl_trigger();
      }
      if constexpr (UPD) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int r = g + 32 * i;
          const float2 d2 = split_f64(prevoff[i] >= 0 ? __ldcg(U.u.delta + r) : 0.0);
          dph[i] = d2.x;
          dpl[i] = d2.y;
        }
      }
      for (int t = 0; t < T; ++t) {
        cp_async_wait<PRE - 1>();  // this thread's copies of stage t have landed
        const uint32_t gt = g0 + (uint32_t)t;  // stage number within the CTA
        const int st = (int)(gt % NS);
        unsigned char* big = raw + st * C::kRawBytes;
        if constexpr (!THREE) {  // the tile is ready for the MMA as loaded
          fence_proxy_async_smem();  // this thread's copies, visible to the tensor core
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[st]);
        }
        if constexpr (UPD) {
          // deferred update of the previous outer step on this stage's 32
          // columns, v_new = v_old - cU * sum_r Yprev[r][k] Delta_r: FP32
          // products and sums (per-thread sums over its rows, a shuffle over
          // the 4 row groups of the warp, one shared-memory exchange between
          // warps; every warp then forms v_new for all 32 columns itself), the
          // subtraction in double-float.  Exact products summed in double-float
          // cost ~35% more time in this pass; the stopping test instead
          // rebuilds v from its definition with exact products before each
          // check (the FP32 roundings then never reach a certificate).
          float up[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            if (prevoff[i] >= 0) {
              const float4 x = *reinterpret_cast<const float4*>(big + C::kPrevOff + dsto[i]);
              up[0] = fmaf(x.x, dph[i], fmaf(x.x, dpl[i], up[0]));
              up[1] = fmaf(x.y, dph[i], fmaf(x.y, dpl[i], up[1]));
              up[2] = fmaf(x.z, dph[i], fmaf(x.z, dpl[i], up[2]));
              up[3] = fmaf(x.w, dph[i], fmaf(x.w, dpl[i], up[3]));
            }
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            up[e] += __shfl_xor_sync(0xffffffffu, up[e], 8);
            up[e] += __shfl_xor_sync(0xffffffffu, up[e], 16);
          }
          // buffer gt & 1 is rewritten at stage gt + 2, after the barrier of
          // stage gt + 1, which every warp reaches after its reads of stage gt
          float* ub = ured + (gt & 1) * (kLoaderWarps * 32);
          if (lane < 8)
            *reinterpret_cast<float4*>(ub + warp * 32 + 4 * l) = make_float4(up[0], up[1], up[2], up[3]);
        }
        // this thread's chunks of the current rows (split products: read here
        // for the conversion; plain TF32: read after the barrier)
        float4 xs[RPT];
        if constexpr (THREE) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) xs[i] = *reinterpret_cast<const float4*>(big + dsto[i]);
        }
        // split products: head / tail tiles into MMA slot gt % MS once the MMA
        // of stage gt - MS has read it; then hand the slot to the MMA.  With
        // two or more MMA slots this runs before the loaders' barrier (the
        // MMA starts while the loaders finish the stage); with one slot it
        // waits for the MMA of the previous stage, so it runs after the
        // projection.
        auto handoff = [&]() {
          if constexpr (THREE) {
            const int ms = (int)(gt % MS);
            // every lane polls the slot's barrier itself (cheaper than one
            // lane waiting and the warp converging on it)
            if (gt >= (uint32_t)MS && ok)
              ok = mbar_wait_bounded(&empty[ms], (uint32_t)((gt / MS - 1) & 1), err);
            unsigned char* hi = mring + ms * C::kMmaSlotBytes;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
              const float4 x = xs[i];
              if constexpr (F16) {
                // x s_r rounded to FP16, 4 columns = 8 bytes (64-byte rows)
                const int r = g + 32 * i;
                const uint32_t off = (uint32_t)((r >> 3) * 512 + (r & 7) * 64 +
                                                ((((l >> 1) ^ ((r >> 1) & 3))) << 4) + (l & 1) * 8);
                const float sc = rsc[i];
                *reinterpret_cast<uint2*>(hi + off) =
                    make_uint2(f16x2_rn(x.x * sc, x.y * sc), f16x2_rn(x.z * sc, x.w * sc));
              } else if constexpr (BF) {
                // x = b0 + b1 (+ a remainder below 2^-16 |x|): bf16 head and
                // tail, 4 columns = 8 bytes, half of a 16-byte chunk of the
                // 64-byte row
                const int r = g + 32 * i;
                const uint32_t off = (uint32_t)((r >> 3) * 512 + (r & 7) * 64 +
                                                ((((l >> 1) ^ ((r >> 1) & 3))) << 4) + (l & 1) * 8);
                const uint32_t h01 = bf16x2_rn(x.x, x.y), h23 = bf16x2_rn(x.z, x.w);
                // the tails x - b0 are exact in FP32
                const uint32_t l01 = bf16x2_rn(x.x - __uint_as_float(h01 << 16),
                                               x.y - __uint_as_float(h01 & 0xFFFF0000u));
                const uint32_t l23 = bf16x2_rn(x.z - __uint_as_float(h23 << 16),
                                               x.w - __uint_as_float(h23 & 0xFFFF0000u));
                *reinterpret_cast<uint2*>(hi + off) = make_uint2(h01, h23);
                *reinterpret_cast<uint2*>(hi + C::kOpTile + off) = make_uint2(l01, l23);
              } else {
                const float4 h = make_float4(tf32_head(x.x), tf32_head(x.y), tf32_head(x.z), tf32_head(x.w));
                *reinterpret_cast<float4*>(hi + dsto[i]) = h;
                *reinterpret_cast<float4*>(hi + C::kOpTile + dsto[i]) =
                    make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
              }
            }
            fence_proxy_async_smem();  // this thread's tiles, visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[ms]);
          }
        };
        if constexpr (THREE && MS >= 2) handoff();
        // every loader's copies of this stage (incl. the v slice) have landed
        // and (fused update) every warp's column sums are in place
        asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
        float vh[4], vl[4];
        if constexpr (UPD) {
          const float* ub = ured + (gt & 1) * (kLoaderWarps * 32);
          float sum = 0.f;  // lane = column
#pragma unroll
          for (int w2 = 0; w2 < kLoaderWarps; ++w2) sum += ub[32 * w2 + lane];
          const float2 vo = reinterpret_cast<const float2*>(vring + (gt % (2 * NS)) * 256)[lane];
          const float2 vn = df_add(vo, df_neg(df_mul(u_cU2, make_float2(sum, 0.f))));
          const long long kk = (U.a0 + t) * 32 + lane;
          if (warp == 0 && kk < U.K) U.u.v2[kk] = vn;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            vh[e] = __shfl_sync(0xffffffffu, vn.x, 4 * l + e);
            vl[e] = __shfl_sync(0xffffffffu, vn.y, 4 * l + e);
          }
        } else {
          // projection vector slice as loaded (exact FP32 pairs)
          const float4* vs = reinterpret_cast<const float4*>(vring + (gt % (2 * NS)) * 256 + l * 32);
          const float4 va = vs[0], vb = vs[1];
          vh[0] = va.x; vh[1] = va.z; vh[2] = vb.x; vh[3] = vb.z;
          vl[0] = va.y; vl[1] = va.w; vl[2] = vb.y; vl[3] = vb.w;
        }
        // projection on this thread's own chunks (exact FP32 inputs)
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          if constexpr (!THREE) xs[i] = *reinterpret_cast<const float4*>(big + dsto[i]);
          const float4 x = xs[i];
          float a = pacc[i];
          a = fmaf(x.x, vh[0], fmaf(x.x, vl[0], a));
          a = fmaf(x.y, vh[1], fmaf(x.y, vl[1], a));
          a = fmaf(x.z, vh[2], fmaf(x.z, vl[2], a));
          a = fmaf(x.w, vh[3], fmaf(x.w, vl[3], a));
          pacc[i] = a;
        }
        if ((t & 7) == 7) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            comp_add(phi[i], plo[i], pacc[i]);
            pacc[i] = 0.f;
          }
        }
        if constexpr (THREE && MS < 2) handoff();
        if constexpr (THREE) {
          // this thread's part of load slot st is consumed: refill it
          if (t + NS < T) issue(t + NS, st);
          cp_async_commit();
        } else {
          // stage gt + NS - 1 into the slot of stage gt - 1 once its MMA completed
          const int tn = t + NS - 1;
          if (ok && tn < T) {
            const uint32_t gn = g0 + (uint32_t)tn;
            const int sn = (int)(gn % NS);
            if (gn >= (uint32_t)NS) ok = warp_wait(&empty[sn], (uint32_t)((gn / NS - 1) & 1), ok);
            if (ok) issue(tn, sn);
          }
          cp_async_commit();
        }
      }
      cp_async_wait<0>();
      // projection partials: reduce over the 8 lanes sharing a row group in
      // double-float (FP64 is slow on this part), one FP64 sum at the end
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        comp_add(phi[i], plo[i], pacc[i]);
        float2 s2 = df_norm(phi[i], plo[i]);
#pragma unroll
        for (int o = 1; o <= 4; o <<= 1)
          s2 = df_add(s2, make_float2(__shfl_xor_sync(0xffffffffu, s2.x, o),
                                      __shfl_xor_sync(0xffffffffu, s2.y, o)));
        if (l == 0) U.ppart[g + 32 * i] = (double)s2.x + (double)s2.y;
      }
      // ---------------- epilogue: TMEM -> FP32 partial tiles ----------------
      ok = warp_wait(done, (uint32_t)(j & 1), ok);
      tc_fence_after();
      // warp w reads TMEM lanes 32 (w % 4) .. +31 (= rows of the M = 128 tile)
      // and the 32-column chunks of parity w / 4
      const int lg = warp & 3, cpar = warp >> 2;
      const int trow = lg * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
      const int n1 = (SBP <= 128) ? ((U.sb + 31) & ~31) : 128;  // MMA N of the first tile
      const int n2 = (U.sb + 31) & ~31;                           // MMA N of rows 128..255
      // partial tiles are stored transposed: entry (row, col) at [col][row], so
      // that the 32 lanes (32 consecutive rows) of a warp write 128 contiguous
      // bytes per column
      float* Pc = U.part;
      if constexpr (F16) {  // every loader's s_rinv entries are in place
        asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
      }
      // scaled FP16: entry (row, col) of the accumulator carries s_row s_col
      auto unscale = [&](float v, int row, int col) {
        if constexpr (F16) return v * s_rinv[row] * s_rinv[col];
        else return v;
      };
      for (int cc = 32 * cpar; cc < n1; cc += 64) {  // rows 0..127, columns 0..n1-1
        uint32_t r[32];
        tmem_ld32(tbase + (uint32_t)cc, r);
        if (cc <= trow && trow < SBP) {  // rows past a short tile hold garbage
#pragma unroll
          for (int q = 0; q < 32; ++q)
            Pc[(long long)(cc + q) * SBP + trow] = unscale(__uint_as_float(r[q]), trow, cc + q);
        }
      }
      if constexpr (SBP == 256) {
        const int grow = 128 + trow;  // rows 128..255, columns 0..n2-1
        for (int cc = 32 * cpar; cc < n2; cc += 64) {
          uint32_t r[32];
          tmem_ld32(tbase + 128u + (uint32_t)cc, r);
          if (cc <= grow) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              Pc[(long long)(cc + q) * SBP + grow] = unscale(__uint_as_float(r[q]), grow, cc + q);
          }
        }
      }
      if (j + 1 < nunits) {
        // the accumulator is read: the MMA may overwrite it with the next
        // unit; every loader is past this unit (s_rinv, ring slots) before
        // the next unit's prologue writes them
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(epi);
        asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
      }
      g0 += (uint32_t)T;
    }
  } else if (lane == 0) {
    // ---------------- MMA issue (one thread) ----------------
    // one K step: 8 tf32 or 16 bf16 = 32 bytes of a row
    auto desc = [](uint32_t a) { return BF ? sw64_kmajor_desc(a) : sw128_kmajor_desc(a); };
    auto mma = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
      if constexpr (BF) mma_bf16(d, a, b, id, acc);
      else mma_tf32(d, a, b, id, acc);
    };
    constexpr int KSTEPS = BF ? 2 : 4;
    constexpr uint32_t kHalf = 128u * C::kOpRow;  // rows 128.. of a 256-row tile
    bool mok = true;
    uint32_t g0 = 0;
    for (int j = 0; j < nunits && mok; ++j) {
      const GramUnitArgs U = unit(j);
      const int T = (int)(U.a1 - U.a0);
      const int n1 = (SBP <= 128) ? ((U.sb + 31) & ~31) : 128;
      const int n2 = (U.sb + 31) & ~31;
      const uint32_t id1 = F16 ? idesc_f16(128, n1) : (BF ? idesc_bf16(128, n1) : idesc_tf32(128, n1));
      const uint32_t id2 = F16 ? idesc_f16(128, n2) : (BF ? idesc_bf16(128, n2) : idesc_tf32(128, n2));
      // the previous unit's accumulator has been read out
      if (j > 0) {
        mok = mbar_wait_bounded(epi, (uint32_t)((j - 1) & 1), err);
        tc_fence_after();
      }
      for (int t = 0; t < T && mok; ++t) {
        const uint32_t gt = g0 + (uint32_t)t;
        int st, lap;
        if constexpr (THREE) {
          st = (int)(gt % MS);
          lap = (int)(gt / MS);
        } else {
          st = (int)(gt % NS);
          lap = (int)(gt / NS);
        }
        if (!mbar_wait_bounded(&full[st], (uint32_t)(lap & 1), err)) {
          mok = false;
          break;
        }
        tc_fence_after();
        const uint32_t hb = THREE ? smem_u32(mring) + (uint32_t)(st * C::kMmaSlotBytes)
                                  : smem_u32(raw) + (uint32_t)(st * C::kRawBytes);
        const uint32_t lb = hb + (uint32_t)C::kOpTile;
#pragma unroll
        for (int kk = 0; kk < KSTEPS; ++kk) {
          const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
          const uint64_t h0 = desc(hb + kk * 32);
          mma(tmem, h0, h0, id1, acc);
          if constexpr (THREE && !F16) {
            const uint64_t l0 = desc(lb + kk * 32);
            mma(tmem, h0, l0, id1, 1u);
            mma(tmem, l0, h0, id1, 1u);
          }
          if constexpr (SBP == 256) {
            const uint64_t h1 = desc(hb + (THREE ? kHalf : 16384u) + kk * 32);
            mma(tmem + 128u, h1, h0, id2, acc);
            if constexpr (THREE && !F16) {
              const uint64_t l0 = desc(lb + kk * 32);
              const uint64_t l1 = desc(lb + kHalf + kk * 32);
              mma(tmem + 128u, h1, l0, id2, 1u);
              mma(tmem + 128u, l1, h0, id2, 1u);
            }
          }
        }
        mma_commit(&empty[st]);
      }
      mma_commit(done);
      g0 += (uint32_t)T;
    }
    // do not release tensor memory before the MMAs are complete
    if (nunits > 0) mbar_wait_bounded(done, (uint32_t)((nunits - 1) & 1), err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
  }
}

template <int SBP, bool THREE, bool UPD, bool PANEL, bool BF, bool F16 = false>
int launch_one(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
               const float2* v2, int P, float* part, double* ppart, unsigned* err,
               const GramUpdate& u, cudaStream_t stream) {
  using C = TcCfg<SBP, THREE, UPD, BF, F16>;
  // the shared-memory limit is a per-device setting: raised once per device
  // and instantiation (a bit per device; setting it twice is harmless)
  static std::atomic<unsigned long long> configured{0ull};
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return (int)ce;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(configured.load(std::memory_order_acquire) & bit)) {
    ce = cudaFuncSetAttribute(k_gram_tc<SBP, THREE, UPD, PANEL, BF, F16, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (ce != cudaSuccess) return (int)ce;
    configured.fetch_or(bit, std::memory_order_release);
  }
  const long long natoms = (K + 31) / 32;
  // launched as a programmatic dependent: its CTAs may start (and prefetch)
  // while the preceding grid in the stream finishes
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::kSmem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_gram_tc<SBP, THREE, UPD, PANEL, BF, F16, false>, A,
                                           lda, N, K, idx, sb, v2, natoms, part, ppart, err, u,
                                           GramBatchArgs{});
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

// Shared launch over several problems (fused update on panels, SBP <= 128).
template <int SBP, bool BF, bool F16, bool THREE>
int launch_batch_one(const GramBatchArgs& bt, int P, unsigned* err, cudaStream_t stream) {
  using C = TcCfg<SBP, THREE, true, BF, F16>;
  auto kern = k_gram_tc<SBP, THREE, true, true, BF, F16, true>;
  static std::atomic<unsigned long long> configured{0ull};
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return (int)ce;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(configured.load(std::memory_order_acquire) & bit)) {
    ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (ce != cudaSuccess) return (int)ce;
    configured.fetch_or(bit, std::memory_order_release);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = C::kSmem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, (const float*)nullptr, 0LL, 0LL, 0LL,
                                           (const int*)nullptr, 0, (const float2*)nullptr, 0LL,
                                           (float*)nullptr, (double*)nullptr, err, GramUpdate{}, bt);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

}  // namespace

int launch_gram_tc_batch(const GramBatchArgs& bt, int P, int sbp, int three_pass, unsigned* err,
                         cudaStream_t stream) {
  // three_pass: 0 = TF32, 1 = 3xTF32, 2 = BF16x3, 3 = scaled FP16
#define CA_TCB_CASE(S)                                                           \
  if (sbp == S) {                                                               \
    if (three_pass == 0) return launch_batch_one<S, false, false, false>(bt, P, err, stream); \
    if (three_pass == 1) return launch_batch_one<S, false, false, true>(bt, P, err, stream);  \
    if (three_pass == 3) return launch_batch_one<S, true, true, true>(bt, P, err, stream);    \
    return launch_batch_one<S, true, false, true>(bt, P, err, stream);                        \
  }
  CA_TCB_CASE(32)
  CA_TCB_CASE(64)
  CA_TCB_CASE(128)
#undef CA_TCB_CASE
  return (int)cudaErrorInvalidValue;
}

int gram_tc_max_sb() { return 256; }

int launch_gram_tc(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
                   const float2* v2, int P, int sbp, float* part, double* ppart, unsigned* err,
                   int three_pass, cudaStream_t stream, const GramUpdate* upd, bool panel) {
  // three_pass: 0 = TF32, 1 = 3xTF32, 2 = BF16x3, 3 = scaled FP16 (needs upd->rscale)
  GramUpdate none{};
  if (upd) {
    none.rscale = upd->rscale;
    none.early = upd->early;
  }
  if (three_pass == 3 && !none.rscale) return (int)cudaErrorInvalidValue;
#define CA_TC_CASE(S, U, PN, UU)                                                              \
  if (sbp == S) {                                                                            \
    if (three_pass == 0)                                                                     \
      return launch_one<S, false, U, PN, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, \
                                                UU, stream);                                 \
    if (three_pass == 1)                                                                     \
      return launch_one<S, true, U, PN, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err,  \
                                               UU, stream);                                  \
    if (three_pass == 3)                                                                     \
      return launch_one<S, true, U, PN, true, true>(A, lda, N, K, idx, sb, v2, P, part, ppart,  \
                                                    err, UU, stream);                        \
    return launch_one<S, true, U, PN, true>(A, lda, N, K, idx, sb, v2, P, part, ppart, err,     \
                                            UU, stream);                                     \
  }
  if (upd && upd->sb > 0) {  // fused deferred update: panels, s*b <= 128 only
    if (!panel || sbp > 128 || upd->sb > sbp) return (int)cudaErrorInvalidValue;
    CA_TC_CASE(32, true, true, *upd)
    CA_TC_CASE(64, true, true, *upd)
    CA_TC_CASE(128, true, true, *upd)
    return (int)cudaErrorInvalidValue;
  }
  if (panel) {
    CA_TC_CASE(32, false, true, none)
    CA_TC_CASE(64, false, true, none)
    CA_TC_CASE(128, false, true, none)
    CA_TC_CASE(256, false, true, none)
  } else {
    CA_TC_CASE(32, false, false, none)
    CA_TC_CASE(64, false, false, none)
    CA_TC_CASE(128, false, false, none)
    CA_TC_CASE(256, false, false, none)
  }
#undef CA_TC_CASE
  return (int)cudaErrorInvalidValue;
}

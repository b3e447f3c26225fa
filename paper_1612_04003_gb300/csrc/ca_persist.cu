// ca_persist.cu -- consecutive outer steps of a dense CA-BCD (Alg. 2) /
// CA-BDCD (Alg. 4) solve on the tensor-core path in one persistent,
// cooperative launch, with the s unrolled solves of step k running while the
// Gram pass of step k+1 already streams its rows.
//
// Per outer step k the solve needs (Sec. 3.1 / 3.2, in the common form of
// the library: A = X or X^T, v = rho or w, x = w or alpha):
//   G_k = Y_k Y_k^T,  p_k = Y_k v_k,  Delta_k from the chain of eq. "recur",
//   v_{k+1} = v_k - cU Y_k^T Delta_k   (the deferred update).
// The Gram G_k needs only the sampled indices; the projection p_k needs v_k,
// i.e. Delta_{k-1}.  Each Gram CTA splits its columns into a region A (its
// first atoms, streamed while the chain of step k-1 still runs) and a region
// B.  In region A, v lags one step further behind:
//   p_k = Y_{k,A} v_{k-1}[A] - cU (Y_{k,A} Y_{k-1,A}^T) Delta_{k-1} + Y_{k,B} v_k[B]
// which is the same sum in exact arithmetic (v_k[A] = v_{k-1}[A] -
// cU Y_{k-1,A}^T Delta_{k-1}).  The cross Gram C = Y_{k,A} Y_{k-1,A}^T comes
// from the current rows and the previous step's rows, both staged, as a
// second tcgen05 accumulator.  Region A's stages also bring in the rows of
// step k-2 and apply that step's deferred update (Delta_{k-2} is known by
// then), so region A's v is v_{k-1} when it is projected; region B applies
// the update of step k-1 first, as the fused Gram pass does.  After the last
// step of a launch, region A gets the update of the step before it, in a
// short final run over its atoms.  The 16-bit operand tiles are written in
// place over the FP32 rows they come from (the load slot holds three row
// sets), and a slot is refilled once the MMA has read it.
//
// Roles (grid = Pg Gram CTAs + 1 chain CTA, one CTA per SM, cooperative so
// that all are resident; every wait is bounded and gives up once any wait of
// the grid has timed out):
//  * Gram CTAs, warps 0-7 (loaders) and warp 8 (TMEM, MMA issue): the passes
//    of steps k0 .. k0+npass-1 over their atom range, one after another with
//    the load ring running across pass boundaries; at the end of a pass they
//    store the FP32 Gram partial and the corrected projection partial and
//    count themselves done (cnt[0]).
//  * Gram CTAs, warps 9-12: once all CTAs finished pass k, they reduce their
//    slice of its partials (CTAs 0 .. s-1: diagonal block j = CTA index,
//    inverted by the sweep operator; the others: 64 lower-triangle or
//    projection entries each) and count themselves done (cnt[1]).
//  * The chain CTA, warps 0-7: once all slices of step k are reduced, the
//    lookahead chain of step k (Delta_k, x updated at the sampled indices),
//    then it publishes Delta_k (cnt[2] = k - k0 + 1).
// The dependencies form no cycle: epilogue k -> reduce k -> chain k ->
// region B of pass k+1 -> epilogue k+1, and every buffer is rewritten only
// after its readers of the previous step have counted themselves done.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "ca_kernels.cuh"
#include "ca_solve.cuh"
#include "ca_tc.cuh"

namespace {

constexpr int kLW = 8;                    // loader warps
constexpr int kLT = 32 * kLW;             // loader threads
constexpr int kMmaW = kLW;                // warp 8
constexpr int kSideW0 = kLW + 1;          // warps 9 .. 12: reduction
constexpr int kSideT = 128;
constexpr int kHalves = kSideT / 64;  // side threads per reduced entry
constexpr int kThreadsP = 32 * kSideW0 + kSideT;  // 416
constexpr int kBarLoad = 1;               // named barriers: loaders (256 threads)
constexpr int kBarSide = 7;               // side warps (128)
constexpr int kBarInv = 8;                // two side warps inverting a block (64)

// MODE: 2 = BF16x3 (bf16 head and tail, three products), 3 = scaled FP16
// (one product of rows multiplied by powers of two)
template <int SBP, int MODE>
struct PCfg {
  static constexpr bool F16 = MODE == 3;
  static constexpr int kTile = SBP * 128;            // SBP rows x 32 FP32
  // load slot: [current | previous | previous-but-one rows], FP32 as loaded;
  // the current rows (and in region A the previous rows) are converted in
  // place into the 16-bit operand tiles the MMA reads (head and tail of 64
  // bytes per row, or one scaled-FP16 tile: the same bytes or fewer)
  static constexpr int kRaw = 3 * kTile;
  static constexpr int kOpTile = SBP * 64;           // 16-bit operand rows of 64 bytes
  static constexpr int kBudget = 200 * 1024;
  static constexpr int kNSfit = kBudget / kRaw;
  static constexpr int kNS = kNSfit < 8 ? kNSfit : 8;
  static constexpr int kRPT = SBP / 32;              // rows per loader thread
  static constexpr int kVRing = 2 * kNS * 256;       // v slices (32 FP32 pairs)
  static constexpr int kUpd = 2 * kLW * 32 * 4;      // column sums of the update, by parity
  static constexpr int kMisc = SBP * 8 + 2 * SBP * 4 + SBP * 8 + 2 * SBP * 4;  // sdl, corr, proj, rinv
  static constexpr int kZero = kNS * kRaw + kVRing + kUpd + kMisc;
  static constexpr int kSmem = kZero + 1024 + 256;
  static constexpr int kTmemCols = 256;               // G at column 0, C at column 128
  static_assert(kNS >= 3, "load ring too shallow");
  static_assert(kSmem <= 232448, "shared memory");
};

// Bounded wait on a count another CTA raises: true once *p >= target; gives
// up (CA_DEV_ERR_TIMEOUT) after the limit or as soon as another wait of the
// grid has given up.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned target, unsigned* err) {
  const uint64_t t0 = ca_globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (*(volatile const unsigned*)p >= target) {
      __threadfence();
      return true;
    }
    if ((it & 63u) == 63u) {
      if (*(volatile unsigned*)err & CA_DEV_ERR_TIMEOUT) return false;
      if (ca_globaltimer() - t0 > CA_WAIT_LIMIT_NS) {
        ca_flag(err, CA_DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// mbarrier wait that also gives up once another wait of the grid has.
__device__ __forceinline__ bool mbar_wait_grid(uint64_t* bar, uint32_t parity, unsigned* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ca_globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u) {
      if (*(volatile unsigned*)err & CA_DEV_ERR_TIMEOUT) return false;
      if (ca_globaltimer() - t0 > CA_WAIT_LIMIT_NS) {
        ca_flag(err, CA_DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async_16_pol(uint32_t dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "l"(pol)
               : "memory");
}

// 4 FP32 values as BF16 head (h) and tail (t) of x = h + t (+ < 2^-16 |x|),
// or (F16) as x * sc rounded to FP16: 8 bytes each.
template <bool F16>
__device__ __forceinline__ void to16(const float4 x, float sc, uint2& h, uint2& t) {
  if constexpr (F16) {
    h = make_uint2(f16x2_rn(x.x * sc, x.y * sc), f16x2_rn(x.z * sc, x.w * sc));
  } else {
    const uint32_t h01 = bf16x2_rn(x.x, x.y), h23 = bf16x2_rn(x.z, x.w);
    h = make_uint2(h01, h23);
    t = make_uint2(bf16x2_rn(x.x - __uint_as_float(h01 << 16), x.y - __uint_as_float(h01 & 0xFFFF0000u)),
                   bf16x2_rn(x.z - __uint_as_float(h23 << 16), x.w - __uint_as_float(h23 & 0xFFFF0000u)));
  }
}

template <int SBP, int MODE>
__global__ void __launch_bounds__(kThreadsP, 1) k_persist(PersistArgs a, unsigned* __restrict__ err) {
  using C = PCfg<SBP, MODE>;
  constexpr bool F16 = C::F16;
  constexpr int NS = C::kNS, RPT = C::kRPT;
  extern __shared__ unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Pg = (int)gridDim.x - 1;
  const int c = blockIdx.x;
  const int sb = a.sb, npass = a.npass;

  // ------------------------------------------------------------ chain CTA
  if (c == Pg) {
    if (warp >= 8) return;
    double* smem_d = reinterpret_cast<double*>(smem_raw);
    for (int p = 0; p < npass; ++p) {
      const long long k = a.k0 + p;
      SolveArgs sa = a.sa;
      sa.idx = a.idx_all + k * sb;
      sa.delta = a.delta2[k & 1];
      chain_la_body<8, 4>(a.Rs, a.pvec, a.Ginv, sa, err, smem_d, a.cnt + 1,
                          (unsigned)(Pg * (p + 1)), false);
      chain_cta_sync();  // Delta_k and x written by every thread of the chain
      if (tid == 0) {
        __threadfence();
        atomicAdd(a.cnt + 2, 1u);
      }
    }
    return;
  }

  // ------------------------------------------------------------ Gram CTA
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* raw = smem;                                  // NS x [cur | prev | prev2 rows]
  unsigned char* vring = raw + NS * C::kRaw;                  // 2 NS x 32 (hi, lo) of v
  float* ured = reinterpret_cast<float*>(vring + C::kVRing);  // [2][kLW][32]
  float2* sdl = reinterpret_cast<float2*>(ured + 2 * kLW * 32);  // Delta_{k-1} (hi, lo)
  float* scorr = reinterpret_cast<float*>(sdl + SBP);        // [2][SBP] correction halves
  float2* sproj = reinterpret_cast<float2*>(scorr + 2 * SBP);  // projection per row
  float* srinv = reinterpret_cast<float*>(sproj + SBP);      // [2][SBP] 1 / row scale, by pass parity
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kZero);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;  // MMA -> epilogue, one phase per pass
  uint64_t* epi = done + 1;     // epilogue -> MMA, one phase per pass
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(epi + 1);

  const long long natoms = a.natoms;
  const long long a0 = natoms * c / Pg, a1 = natoms * (c + 1) / Pg;
  const int T = (int)(a1 - a0);
  const int NA = a.na < T ? a.na : T;  // region-A atoms of the passes after the first
  // T stages per pass, then (two passes or more) the deferred update of the
  // region-A atoms for the last pass's previous step
  const long long S_tot = (long long)npass * T + (npass >= 2 ? NA : 0);
  const long long N = a.N;

  if (tid == 0) {
    for (int s2 = 0; s2 < NS; ++s2) {
      mbar_init(&full[s2], kLT);  // one arrival per loader thread
      mbar_init(&empty[s2], 1);
    }
    mbar_init(done, 1);
    mbar_init(epi, kLW);
    fence_mbar_init();
  }
  if (warp == kMmaW) {
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

  if (warp < kLW) {
    // ---------------- loaders / projection / update / epilogue ----------------
    // Stages of this CTA in order: pass p = 0 .. npass-1, atom a0 + t for
    // t < T (region A: p > 0, t < NA), then (npass >= 2) the deferred update
    // of region-A atom a0 + t, t < NA, for the last pass's previous step.
    const int g = tid >> 3, l = tid & 7;
    uint32_t dsto[RPT], opoff[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = g + 32 * i;
      dsto[i] = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((l ^ (r & 7)) << 4));
      opoff[i] = (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((l >> 1) ^ ((r >> 1) & 3))) << 4) +
                            (l & 1) * 8);
    }
    const uint32_t raw0 = smem_u32(raw), vring0 = smem_u32(vring);
    const uint64_t pol_stream = l2_evict_first();
    bool ok = true;
    auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
      bool r = ok;
      if (lane == 0 && r) r = mbar_wait_grid(bar, parity, err);
      r = __shfl_sync(0xffffffffu, r ? 1 : 0, 0) != 0;
      __syncwarp();
      ok = r;
    };
    // issue side: this thread's rows (row index or -1) of the pass being
    // issued (icur), its previous step (iprv) and the one before (iprv2);
    // every stage of a pass is issued before the first of the next
    int icur[RPT], iprv[RPT], iprv2[RPT];
    auto load_rows = [&](const int* idx, int nsb, int (&out)[RPT]) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = g + 32 * i;
        int gi = r < nsb ? idx[r] : -1;
        if (r < nsb && (gi < 0 || gi >= N)) {
          ca_flag(err, CA_DEV_ERR_ARG);
          gi = -1;
        }
        out[i] = gi;
      }
    };
    load_rows(a.prev_idx, a.prev_sb, icur);  // "pass -1"
#pragma unroll
    for (int i = 0; i < RPT; ++i) iprv[i] = -1;
    int ip = 0, itp = 0;  // position of the next stage to issue
    auto issue = [&](long long gs, int slot) {
      const int p = ip, t = itp;
      if (++itp == T) {
        ++ip;
        itp = 0;
      }
      const bool fin = p == npass;  // the final deferred update of region A
      if (t == 0 && !fin) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          iprv2[i] = iprv[i];
          iprv[i] = icur[i];
        }
        load_rows(a.idx_all + (a.k0 + p) * sb, sb, icur);
      }
      const bool regA2 = !fin && p >= 2 && t < NA;  // region A with the lagged update
      const long long atom = a0 + t;
      const uint32_t dst = raw0 + (uint32_t)(slot * C::kRaw);
      const float* base = a.A + atom * N * 32 + 4 * l;
      if (!fin) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (icur[i] >= 0) cp_async_16_pol(dst + dsto[i], base + (long long)icur[i] * 32, pol_stream);
      }
#pragma unroll
      for (int i = 0; i < RPT; ++i)
        if (iprv[i] >= 0)
          cp_async_16_pol(dst + C::kTile + dsto[i], base + (long long)iprv[i] * 32, pol_stream);
      if (regA2) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (iprv2[i] >= 0)
            cp_async_16_pol(dst + 2 * C::kTile + dsto[i], base + (long long)iprv2[i] * 32, pol_stream);
      }
      if (tid < 16)  // the stage's 32 (hi, lo) pairs of v
        cp_async_16_zfill(vring0 + (uint32_t)((gs % (2 * NS)) * 256 + tid * 16),
                          a.v2 + atom * 32 + 2 * tid, 16u);
    };
    // NS - 1 stages in flight: a slot is refilled once its MMA has read the
    // tiles converted in place, one stage after it was consumed
    constexpr int LAG = 1;  // a slot is refilled one stage after its consumption
    for (int t = 0; t < NS - LAG; ++t) {
      if (t < S_tot) issue(t, t);
      cp_async_commit();
    }
    const float2 cU2 = split_f64(a.cU);
    int vprev[RPT], vprev2[RPT];  // this thread's rows of steps k-1, k-2 (row index or -1)
    float dph[RPT], dpl[RPT];     // Delta_{k-1} of those rows (hi, lo)
    float dph2[RPT], dpl2[RPT];   // Delta_{k-2}
    float rsc[RPT], rscp[RPT];    // scaled FP16: row multipliers (current, previous)
    float pacc[RPT], phi[RPT], plo[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      vprev[i] = vprev2[i] = -1;
      dph[i] = dpl[i] = dph2[i] = dpl2[i] = 0.f;
    }
    long long gs = 0;        // stages consumed so far (= Gram stages until the final update)
    bool prev_gram = false;  // the previous stage's slot holds tiles the MMA reads
    bool prev_gram2 = false;  // ... the stage before it
    auto load_delta = [&](const double* dl, int psb) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = g + 32 * i;
        const float2 d2 = split_f64((vprev[i] >= 0 && r < psb) ? __ldcg(dl + r) : 0.0);
        dph[i] = d2.x;
        dpl[i] = d2.y;
      }
      for (int q = tid; q < SBP; q += kLT) sdl[q] = split_f64(q < psb ? __ldcg(dl + q) : 0.0);
    };
    // One stage of atom a0 + t.  KIND 0: region A of the second pass (current
    // rows, previous rows as the cross Gram's operand, projection on v as
    // loaded); 1: region A of later passes (as 0, and first the deferred
    // update of the step before the previous one, from its rows); 2: region B
    // (the deferred update of the previous step first, projection on the
    // updated v); 3: region B of a first step (no update); 4: the final
    // deferred update of a region-A atom.  Each kind is straight-line code:
    // the loop is bound by its latency, and a branch per stage costs time.
    auto stage = [&](auto kind, int t) {
      constexpr int KIND = decltype(kind)::value;
      constexpr bool GRAM = KIND <= 3, REGA = KIND <= 1, UPD = KIND == 1 || KIND == 2 || KIND == 4;
      constexpr int UOFF = KIND == 1 ? 2 * C::kTile : C::kTile;  // rows of the update
      cp_async_wait<NS - LAG - 1>();  // this thread's copies of stage gs have landed
      const int st = (int)(gs % NS);
      unsigned char* big = raw + st * C::kRaw;
      if constexpr (UPD) {
        // v_new = v_old - cU sum_r Y[r][k] Delta_r on the stage's 32 columns:
        // FP32 products and sums, the subtraction in double-float (the drift
        // this leaves in v is removed wherever v is rebuilt)
        float up[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int vr = KIND == 1 ? vprev2[i] : vprev[i];
          const float dh = KIND == 1 ? dph2[i] : dph[i], dlo = KIND == 1 ? dpl2[i] : dpl[i];
          if (vr >= 0) {
            const float4 x = *reinterpret_cast<const float4*>(big + UOFF + dsto[i]);
            up[0] = fmaf(x.x, dh, fmaf(x.x, dlo, up[0]));
            up[1] = fmaf(x.y, dh, fmaf(x.y, dlo, up[1]));
            up[2] = fmaf(x.z, dh, fmaf(x.z, dlo, up[2]));
            up[3] = fmaf(x.w, dh, fmaf(x.w, dlo, up[3]));
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          up[e] += __shfl_xor_sync(0xffffffffu, up[e], 8);
          up[e] += __shfl_xor_sync(0xffffffffu, up[e], 16);
        }
        float* ub = ured + (gs & 1) * (kLW * 32);
        if (lane < 8)
          *reinterpret_cast<float4*>(ub + warp * 32 + 4 * l) = make_float4(up[0], up[1], up[2], up[3]);
      }
      float4 xs[RPT], xp[RPT];
      if constexpr (GRAM) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) xs[i] = *reinterpret_cast<const float4*>(big + dsto[i]);
      }
      if constexpr (REGA) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          xp[i] = vprev[i] >= 0 ? *reinterpret_cast<const float4*>(big + C::kTile + dsto[i])
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      // every loader has read its FP32 chunks of this stage (the tiles below
      // overwrite them) and written its column sums; every copy (v slice
      // included) has landed
      asm volatile("bar.sync %0, %1;" ::"n"(kBarLoad), "n"(kLT) : "memory");
      if constexpr (GRAM) {
        // operand tiles in place: current rows at the slot's start, region A's
        // previous rows where they were loaded
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          uint2 h, tl;
          to16<F16>(xs[i], F16 ? rsc[i] : 1.f, h, tl);
          *reinterpret_cast<uint2*>(big + opoff[i]) = h;
          if constexpr (!F16) *reinterpret_cast<uint2*>(big + C::kOpTile + opoff[i]) = tl;
        }
        if constexpr (REGA) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            uint2 h, tl;
            to16<F16>(xp[i], F16 ? rscp[i] : 1.f, h, tl);
            *reinterpret_cast<uint2*>(big + C::kTile + opoff[i]) = h;
            if constexpr (!F16) *reinterpret_cast<uint2*>(big + C::kTile + C::kOpTile + opoff[i]) = tl;
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(&full[st]);  // every loader thread arrives (count 256)
      }
      // refill the slot of stage gs - 1 (consumed; its tiles read by the MMA)
      if (gs + NS - LAG < S_tot) {
        const int ps = (int)((gs + NS - LAG) % NS);
        const bool was_gram = LAG == 1 ? prev_gram : prev_gram2;
        // every lane polls the slot's barrier itself: cheaper than one lane
        // waiting and the warp converging on it (measured ~3% a solve)
        if (gs >= LAG && was_gram && ok)
          ok = mbar_wait_grid(&empty[ps], (uint32_t)(((gs - LAG) / NS) & 1), err);
        issue(gs + NS - LAG, ps);
      }
      cp_async_commit();
      prev_gram2 = prev_gram;
      prev_gram = GRAM;
      float vh[4], vl[4];
      if constexpr (UPD) {
        const float* ub = ured + (gs & 1) * (kLW * 32);
        float sum = 0.f;  // lane = column
#pragma unroll
        for (int w2 = 0; w2 < kLW; ++w2) sum += ub[32 * w2 + lane];
        const float2 vo = reinterpret_cast<const float2*>(vring + (gs % (2 * NS)) * 256)[lane];
        const float2 vn = df_add(vo, df_neg(df_mul(cU2, make_float2(sum, 0.f))));
        const long long col = (a0 + t) * 32 + lane;
        if (warp == 0 && col < a.K) a.v2[col] = vn;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          vh[e] = __shfl_sync(0xffffffffu, vn.x, 4 * l + e);
          vl[e] = __shfl_sync(0xffffffffu, vn.y, 4 * l + e);
        }
      } else {
        const float4* vs = reinterpret_cast<const float4*>(vring + (gs % (2 * NS)) * 256 + l * 32);
        const float4 va = vs[0], vb = vs[1];
        vh[0] = va.x; vh[1] = va.z; vh[2] = vb.x; vh[3] = vb.z;
        vl[0] = va.y; vl[1] = va.w; vl[2] = vb.y; vl[3] = vb.w;
      }
      if constexpr (GRAM) {  // projection on this thread's chunks
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const float4 x = xs[i];
          float s = pacc[i];
          s = fmaf(x.x, vh[0], fmaf(x.x, vl[0], s));
          s = fmaf(x.y, vh[1], fmaf(x.y, vl[1], s));
          s = fmaf(x.z, vh[2], fmaf(x.z, vl[2], s));
          s = fmaf(x.w, vh[3], fmaf(x.w, vl[3], s));
          pacc[i] = s;
        }
        if ((t & 7) == 7) {
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            comp_add(phi[i], plo[i], pacc[i]);
            pacc[i] = 0.f;
          }
        }
      }
      ++gs;
    };
    // end of pass p: Gram partial (TMEM -> FP32 tile), projection partial
    // corrected by C Delta_{k-1} (region A), count this CTA done
    auto epilogue = [&](int p, int psb, int nap) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        comp_add(phi[i], plo[i], pacc[i]);
        pacc[i] = 0.f;
        float2 s2 = df_norm(phi[i], plo[i]);
#pragma unroll
        for (int o = 1; o <= 4; o <<= 1)
          s2 = df_add(s2, make_float2(__shfl_xor_sync(0xffffffffu, s2.x, o),
                                      __shfl_xor_sync(0xffffffffu, s2.y, o)));
        if (l == 0) sproj[g + 32 * i] = s2;
      }
      warp_wait(done, (uint32_t)(p & 1));
      tc_fence_after();
      const int lg = warp & 3, cpar = warp >> 2;
      const int trow = lg * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
      const int nG = (sb + 31) & ~31;
      float* Pc = a.part + (long long)c * SBP * SBP;
      const float* rinv = srinv + (p & 1) * SBP;
      const float* pinv = srinv + ((p + 1) & 1) * SBP;
      for (int cc = 32 * cpar; cc < nG; cc += 64) {
        uint32_t r[32];
        tmem_ld32(tbase + (uint32_t)cc, r);
        if (cc <= trow && trow < SBP) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            float vq = __uint_as_float(r[q]);
            if constexpr (F16) vq *= rinv[trow] * rinv[cc + q];
            Pc[(long long)(cc + q) * SBP + trow] = vq;
          }
        }
      }
      float corr = 0.f;
      if (nap > 0) {  // C Delta_{k-1}, row trow (this warp's half of the columns)
        const int nC = (psb + 31) & ~31;
        for (int cc = 32 * cpar; cc < nC; cc += 64) {
          uint32_t r[32];
          tmem_ld32(tbase + 128u + (uint32_t)cc, r);
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            float vq = __uint_as_float(r[q]);
            if constexpr (F16) vq *= pinv[cc + q];
            const float2 d = sdl[cc + q];
            corr = fmaf(vq, d.x, fmaf(vq, d.y, corr));
          }
        }
        if constexpr (F16) corr *= rinv[trow];
      }
      if (trow < SBP) scorr[cpar * SBP + trow] = corr;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(epi);  // the accumulators are read
      asm volatile("bar.sync %0, %1;" ::"n"(kBarLoad), "n"(kLT) : "memory");
      if (tid < sb) {
        const float2 s2 = sproj[tid];
        const double cr = (double)scorr[tid] + (double)scorr[SBP + tid];
        a.ppart[(long long)c * SBP + tid] = ((double)s2.x + (double)s2.y) - a.cU * cr;
      }
      asm volatile("bar.sync %0, %1;" ::"n"(kBarLoad), "n"(kLT) : "memory");
      if (tid == 0) {
        __threadfence();
        atomicAdd(a.cnt + 0, 1u);
      }
    };
    using KA1 = std::integral_constant<int, 0>;
    using KA2 = std::integral_constant<int, 1>;
    using KB = std::integral_constant<int, 2>;
    using KB0 = std::integral_constant<int, 3>;
    using KT = std::integral_constant<int, 4>;
    for (int p = 0; p < npass; ++p) {
      const long long k = a.k0 + p;
      const int psb = p == 0 ? a.prev_sb : sb;
      const int nap = p == 0 ? 0 : NA;  // region-A atoms of this pass
      const int* idx = a.idx_all + k * sb;
      const int* pidx = p == 0 ? a.prev_idx : a.idx_all + (k - 1) * sb;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = g + 32 * i;
        // step k-2 is what the previous pass called its previous step
        vprev2[i] = vprev[i];
        dph2[i] = dph[i];
        dpl2[i] = dpl[i];
        vprev[i] = (r < psb && pidx[r] >= 0 && pidx[r] < N) ? pidx[r] : -1;
        pacc[i] = phi[i] = plo[i] = 0.f;
        if constexpr (F16) {
          const int gi = (r < sb && idx[r] >= 0 && idx[r] < N) ? idx[r] : -1;
          rscp[i] = vprev[i] >= 0 ? __ldg(a.rscale + vprev[i]) : 1.f;
          rsc[i] = gi >= 0 ? __ldg(a.rscale + gi) : 1.f;
          if (l == 0) srinv[(p & 1) * SBP + r] = 1.f / rsc[i];
          if (l == 0 && p == 0) srinv[SBP + r] = 1.f / rscp[i];
        }
      }
      if (p == 0 && psb > 0) load_delta(a.delta2[(k - 1) & 1], psb);  // written before this launch
      if (p == 1) {
        for (int t = 0; t < nap; ++t) stage(KA1{}, t);
      } else {
        for (int t = 0; t < nap; ++t) stage(KA2{}, t);
      }
      if (p > 0) {  // Delta_{k-1}: the chain of step k-1 in this launch
        if (lane == 0 && ok) ok = wait_count(a.cnt + 2, (unsigned)p, err);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        load_delta(a.delta2[(k - 1) & 1], psb);
        // sdl complete before any warp's epilogue reads it (region B may be empty)
        asm volatile("bar.sync %0, %1;" ::"n"(kBarLoad), "n"(kLT) : "memory");
      }
      if (psb > 0) {
        for (int t = nap; t < T; ++t) stage(KB{}, t);
      } else {
        for (int t = nap; t < T; ++t) stage(KB0{}, t);
      }
      epilogue(p, psb, nap);
    }
    // region A still lacks the update of the last pass's previous step
    if (npass >= 2)
      for (int t = 0; t < NA; ++t) stage(KT{}, t);
    cp_async_wait<0>();
  } else if (warp == kMmaW) {
    // ---------------- MMA issue (one thread) ----------------
    if (lane == 0) {
      bool mok = true;
      uint32_t mg = 0;
      for (int p = 0; p < npass && mok; ++p) {
        const int psb = p == 0 ? a.prev_sb : sb;
        const int nG = (sb + 31) & ~31, nC = (psb + 31) & ~31;
        const uint32_t idG = F16 ? idesc_f16(128, nG) : idesc_bf16(128, nG);
        const uint32_t idC = F16 ? idesc_f16(128, nC > 0 ? nC : 32) : idesc_bf16(128, nC > 0 ? nC : 32);
        if (p > 0) {  // the epilogue has read the previous pass's accumulators
          mok = mbar_wait_grid(epi, (uint32_t)((p - 1) & 1), err);
          tc_fence_after();
        }
        for (int t = 0; t < T && mok; ++t, ++mg) {
          const int ms = (int)(mg % NS);  // the load slot holding the stage's tiles
          if (!mbar_wait_grid(&full[ms], (uint32_t)((mg / NS) & 1), err)) {
            mok = false;
            break;
          }
          tc_fence_after();
          const bool regA = p > 0 && t < NA;
          const uint32_t cb = smem_u32(raw) + (uint32_t)(ms * C::kRaw);
          const uint32_t pb = cb + (uint32_t)C::kTile;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {  // two K = 16 steps of 16-bit values per stage
            const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
            const uint64_t ch = sw64_kmajor_desc(cb + kk * 32);
            if constexpr (F16) {
              mma_bf16(tmem, ch, ch, idG, acc);
              if (regA) mma_bf16(tmem + 128u, ch, sw64_kmajor_desc(pb + kk * 32), idC, acc);
            } else {
              const uint64_t cl = sw64_kmajor_desc(cb + C::kOpTile + kk * 32);
              mma_bf16(tmem, ch, ch, idG, acc);
              mma_bf16(tmem, ch, cl, idG, 1u);
              mma_bf16(tmem, cl, ch, idG, 1u);
              if (regA) {
                const uint64_t ph = sw64_kmajor_desc(pb + kk * 32);
                const uint64_t pl = sw64_kmajor_desc(pb + C::kOpTile + kk * 32);
                mma_bf16(tmem + 128u, ch, ph, idC, acc);
                mma_bf16(tmem + 128u, ch, pl, idC, 1u);
                mma_bf16(tmem + 128u, cl, ph, idC, 1u);
              }
            }
          }
          mma_commit(&empty[ms]);
        }
        mma_commit(done);
      }
      if (npass > 0) mbar_wait_grid(done, (uint32_t)((npass - 1) & 1), err);
    }
  } else {
    // ---------------- side warps: reduction of each step's partials ----------------
    __shared__ float2 red2[kSideT];
    __shared__ double redp[kSideT];
    __shared__ float2 Mb[64];
    __shared__ float2 colbuf[66];
    const int st = tid - 32 * kSideW0;  // 0 .. 127
    const int b = a.sa.b, ndiag = a.sa.s_cur;
    const long long sq = (long long)SBP * SBP;
    const int ldr = a.sa.ldr;
    const float2 cG2 = split_f64(a.sa.cG), cI2 = split_f64(a.sa.cI);
    const long long nlow = (long long)sb * (sb + 1) / 2;
    const int ncta = Pg - ndiag;
    bool sok = true;
    for (int p = 0; p < npass; ++p) {
      if (st == 0 && sok) sok = wait_count(a.cnt + 0, (unsigned)(Pg * (p + 1)), err);
      asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
      if (c < ndiag) {
        // diagonal block c: thread st sums entry (i, jc) over partials of parity st / 64
        const int base = c * b;
        const int e = st & 63, i = e & 7, jc = e >> 3, half = st >> 6;  // (half < kHalves)
        red2[st] = (i < b && jc < b && i >= jc)
                       ? sum_partials<float, 40>(a.part + (long long)(base + jc) * SBP + (base + i),
                                                 half, Pg, kHalves, sq)
                       : make_float2(0.f, 0.f);
        asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
        if (st < 64 && i < b && jc < b && i >= jc) {
          const float2 tt = kHalves > 1 ? df_add(red2[st], red2[st + 64]) : red2[st];
          float2 v = df_mul(cG2, tt);
          if (i == jc) v = df_add(v, cI2);
          Mb[i * b + jc] = v;
          Mb[jc * b + i] = v;
        }
        asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
        if (st < 64) {
          float2 av[1] = {st < b * b ? Mb[st] : make_float2(0.f, 0.f)};
          cta_sweep_inverse<1, 64, kBarInv>(av, b, colbuf, a.Ginv + (long long)c * b * b, err, st);
        }
      } else {
        const int ent = st & 63, half = st >> 6;
        for (long long e0 = (long long)(c - ndiag) * 64; e0 < nlow + sb; e0 += (long long)ncta * 64) {
          const long long e = e0 + ent;
          int i = 0, j = 0, kind = 0;
          float2 s2 = make_float2(0.f, 0.f);
          double sp = 0.0;
          if (e < nlow) {
            int ir, jr;
            tri_decode(e, ir, jr);
            i = sb - 1 - jr;
            j = sb - 1 - ir;
            kind = 1;
            s2 = sum_partials<float, 40>(a.part + (long long)j * SBP + i, half, Pg, kHalves, sq);
          } else if (e < nlow + sb) {
            kind = 2;
            i = (int)(e - nlow);
            const float2 q = sum_partials<double, 40>(a.ppart + i, half, Pg, kHalves, (long long)SBP);
            sp = (double)q.x + (double)q.y;
          }
          red2[st] = s2;
          redp[st] = sp;
          asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
          if (half == 0 && kind == 1) {
            const float2 tt = kHalves > 1 ? df_add(red2[ent], red2[ent + 64]) : red2[ent];
            a.R[(long long)i * ldr + j] = (double)tt.x + (double)tt.y;
            a.Rs[(long long)j * ldr + i] = df_mul(cG2, tt);
          } else if (half == 0 && kind == 2) {
            a.pvec[i] = kHalves > 1 ? redp[ent] + redp[ent + 64] : redp[ent];
          }
          asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
        }
      }
      asm volatile("bar.sync %0, %1;" ::"n"(kBarSide), "n"(kSideT) : "memory");
      if (st == 0) {
        __threadfence();
        atomicAdd(a.cnt + 1, 1u);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaW) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
  }
}

template <int SBP, int MODE>
int launch_persist_one(const PersistArgs& a, int grid, unsigned* err, cudaStream_t stream) {
  using C = PCfg<SBP, MODE>;
  // the chain CTA's shared memory fits in the Gram CTAs' (the same launch)
  const int smem = C::kSmem;
  if ((int)a.chain_smem > smem) return (int)cudaErrorInvalidValue;
  static std::atomic<unsigned long long> configured{0ull};
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return (int)ce;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(configured.load(std::memory_order_acquire) & bit)) {
    ce = cudaFuncSetAttribute(k_persist<SBP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              C::kSmem);
    if (ce != cudaSuccess) return (int)ce;
    configured.fetch_or(bit, std::memory_order_release);
  }
  int per_sm = 0;
  ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<SBP, MODE>, kThreadsP, smem);
  if (ce != cudaSuccess) return (int)ce;
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreadsP);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_persist<SBP, MODE>, a, err);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

}  // namespace

int persist_load_ring(int sbp, int mode) {
  if (mode == 2) return sbp == 32 ? PCfg<32, 2>::kNS : sbp == 64 ? PCfg<64, 2>::kNS : PCfg<128, 2>::kNS;
  return sbp == 32 ? PCfg<32, 3>::kNS : sbp == 64 ? PCfg<64, 3>::kNS : PCfg<128, 3>::kNS;
}

int launch_persist(const PersistArgs& a, int grid, int sbp, int mode, unsigned* err,
                   cudaStream_t stream) {
  // mode: 2 = BF16x3, 3 = scaled FP16
#define CA_P_CASE(S)                                                           \
  if (sbp == S) {                                                             \
    if (mode == 2) return launch_persist_one<S, 2>(a, grid, err, stream);     \
    if (mode == 3) return launch_persist_one<S, 3>(a, grid, err, stream);     \
  }
  CA_P_CASE(32)
  CA_P_CASE(64)
  CA_P_CASE(128)
#undef CA_P_CASE
  return (int)cudaErrorInvalidValue;
}

// Spread of the 2D adjoint on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators), float32, W = 8 taps, 2b = 8 boundary columns, 16 x 16 tiles.
//
// For one work item (tile (bx, by), samples s0..s1) every output of the spread
// (Sec. 3.2 adjoint NDFT with the App. C boundary terms) is a sum over the
// item's samples of outer products (v = u conj(wx wy), v0_k = u conj(wy)
// conj(bx_k), v1_k = u conj(wx) conj(by_k), A_k = u conj(bx_k)):
//   P[x][y]    += (v wx[x - px]) wy[y - py]     interior (24 x 24 padded tile)
//   S0[k][y]   += v0_k wy[y - py]               x-sides
//   S1[k][x]   += v1_k wx[x - px]               y-sides
//   Cc[kx][ky] += A_kx conj(by_ky)              corners
// i.e. two GEMMs with K = samples, D1 = A1 B1^T and D2 = A2 B2^T:
//   A1 (128 rows): [Re v wx (24) | Im v wx (24) | Re v0 (8) | Im v0 (8)] hi, then lo
//   B1 ( 48 rows): [wy (24)] hi, then lo
//   A2 ( 64 rows): [Re v1 | Im v1 | Re A | Im A] (8 each) hi, then lo
//   B2 ( 80 rows): [wx (24) | Re conj(by) (8) | Im conj(by) (8)] hi, then lo
// Every operand value x is split x = hi + lo (hi: x rounded to TF32, lo: the
// exact float32 remainder), so one kind::tf32 MMA over the stacked hi/lo rows
// and columns yields the four products hi*hi, hi*lo, lo*hi, lo*lo in separate
// blocks of D; the epilogue adds the first three (the 3xTF32 scheme, ~21
// significant bits per product, float32-level accuracy).
//
// Pipeline (one CTA of 4 warps per work item, batches of 16 samples = two K = 8
// steps; operands double-buffered in shared memory, K-major without swizzle):
//   staging  cp.async copies the next batch's per-sample inputs while this batch
//            is built;
//   build    each warp takes 4 samples, lane (sample, index a) writes the
//            sample's tap a / boundary index a entries of the four operands
//            (conflict-free: the 8 rows x 4 samples of one warp store fall in 32
//            distinct banks); window entries of the sample that held the slot
//            two batches ago are cleared first, so the operands stay zero
//            elsewhere;
//   MMA      one thread issues tcgen05.mma for both GEMMs and both K steps and
//            commits them to the buffer's mbarrier; the build of the batch after
//            next waits on that mbarrier before it overwrites the buffer;
//   epilogue tcgen05.ld of D1 (TMEM columns 80..127) and D2 (0..79), hi/lo terms
//            combined across warps through shared memory, the partial tile
//            written with 16-byte stores in the layout of k_spread2d.
// Every mbarrier wait is bounded (about one second of clock64); on expiry the
// kernel sets *err, waits once more (bounded) for its MMAs, frees its TMEM and
// returns without writing its partial tile.
#pragma once

#include <stdint.h>

namespace gs {
namespace dev {
namespace tc5 {

constexpr int SB = 16;  // samples per batch (the K of one round: two K = 8 MMA steps)
constexpr int W = 8, B2 = 8, TILE = 16, PW = TILE + W;
constexpr int GRP = SB / 4 * 32;  // floats per 8-row core-matrix group: all K of a batch (SBO = 4 GRP bytes)
constexpr int SBO_BYTES = GRP * 4;
constexpr int LBO_BYTES = 128;    // next 4-element K core matrix
// operand buffer (floats): A1 | B1 | A2 | B2.  MMA-2 runs with M = 128: its rows
// 64..127 fall on B2 (inside the buffer); those rows of D2 are never read.
constexpr int O_A1 = 0, O_B1 = O_A1 + 16 * GRP, O_A2 = O_B1 + 6 * GRP, O_B2 = O_A2 + 8 * GRP;
constexpr int BUF = O_B2 + 10 * GRP;
static_assert(O_A2 + 16 * GRP <= BUF, "rows 64..127 of the second A operand must stay inside the buffer");
// staging, per buffer (floats)
constexpr int S_WIN = 0;                // [SB][24]: x taps 0..7, y taps 8..15
constexpr int S_BX = S_WIN + SB * 24;   // [SB][16]: 8 complex x-boundary factors
constexpr int S_BY = S_BX + SB * 16;    // [SB][16]
constexpr int S_W = S_BY + SB * 16;     // [SB][4]: wx re, im, wy re, im
constexpr int S_U = S_W + SB * 4;       // [SB][2]
constexpr int S_FL = S_U + SB * 2;      // [SB][2] int
constexpr int S_SIZE = S_FL + SB * 2;
constexpr int NBUF = 2;    // operand buffers: the build of batch b waits for the MMAs of batch b - NBUF
constexpr int STAGES = 3;  // staging buffers: batch b + 2 is copied while batch b is built
constexpr int O_STAGE = NBUF * BUF;
constexpr int O_BAR = O_STAGE + STAGES * S_SIZE;  // NBUF mbarriers (8 bytes each), TMEM base, abort flag
constexpr int N_SMEM = O_BAR + 2 * NBUF + 2;
static_assert(O_STAGE % 4 == 0 && S_SIZE % 4 == 0 && O_BAR % 2 == 0, "16-byte staging, 8-byte mbarriers");
// epilogue areas (reuse the operand buffers once every MMA has completed)
constexpr int PART = PW * PW + 2 * B2 * PW + B2 * B2;  // complex values of the partial tile
constexpr int LX = 25, LZ = 41;                        // padded row strides
constexpr int E_H = 0, E_X = E_H + 64 * LX, E_Y = E_X + 64 * LX, E_Z = E_Y + 32 * LZ;
static_assert(E_Z + 32 * LZ <= NBUF * BUF, "epilogue must fit the operand area");
// TMEM columns
constexpr uint32_t TM_D2 = 0, TM_D1 = 80, TM_COLS = 128;
constexpr uint32_t idesc_tf32(int M, int N) {  // D f32, A and B tf32, both K-major
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t ID1 = idesc_tf32(128, 48), ID2 = idesc_tf32(128, 80);

// float offset of element (row r, column k) of an operand: K-major core matrices
// of 8 rows x 16 bytes, K-adjacent ones 128 bytes apart, 8-row groups GRP apart
__device__ __forceinline__ int eo(int r, int k) { return (r >> 3) * GRP + (k >> 2) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start, LBO, SBO (>> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(LBO_BYTES >> 4) << 16) | ((uint64_t)(SBO_BYTES >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{.reg .pred p; setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
// named barriers: id 1 + q, the operands of buffer q are built (4 builder warps
// arrive, the MMA warp waits); id NB_BUILD, the builder warps among themselves
__device__ __forceinline__ void nb_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nb_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
constexpr int NB_BUILD = 1 + NBUF, BUILDERS = 128, THREADS = 160;
// bounded wait for the completion of the mbarrier phase with this parity
__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (true) {
    asm volatile(
        "{.reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q;}\n"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 8 consecutive TMEM columns of this warp's 32 lanes (thread = lane)
__device__ __forceinline__ void tld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
// x = hi + lo, hi rounded to TF32 (10 explicit mantissa bits), lo exact in float32
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
  lo = x - hi;
}
// the hi part of x at row rh, the lo part at row rl, column k
__device__ __forceinline__ void put2(float* op, int rh, int rl, int k, float x) {
  float hi, lo;
  split(x, hi, lo);
  op[eo(rh, k)] = hi;
  op[eo(rl, k)] = lo;
}
__device__ __forceinline__ void cp16(float* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src));
}
__device__ __forceinline__ void cp8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr(dst)), "l"(src));
}
__device__ __forceinline__ void cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr(dst)), "l"(src));
}

// Copies the inputs of samples sb .. sb+nb-1 to a staging buffer; thread t
// takes sample j = t % 16 and part t / 16 of its inputs.  Part 6 copies the
// sample value u[ui] (ui: the sample's index in the caller's order, loaded one
// batch ahead by the caller).
constexpr int PART_U = 6;
__device__ __forceinline__ void stage(float* sg, int tid, int sb, int nb, const float* __restrict__ win,
                                      const float2* __restrict__ w, const float2* __restrict__ bf,
                                      const float2* __restrict__ u, int ui,
                                      const int32_t* __restrict__ fl, int64_t M, bool with_u = true) {
  const int j = tid & (SB - 1), part = tid >> 4;
  if (j >= nb) return;
  const int64_t s = sb + j;
  switch (part) {
    case 0:
    case 1: {  // x taps (part 0), y taps (part 1)
      const float* src = win + s * (2 * W) + part * W;
      cp16(sg + S_WIN + j * 24 + part * W, src);
      cp16(sg + S_WIN + j * 24 + part * W + 4, src + 4);
    } break;
    case 2:
    case 3:
    case 4:
    case 5: {  // boundary factors: x (parts 2, 3), y (parts 4, 5), two 16-byte chunks each
      const int dim = (part >= 4), h = (part & 1);
      const float2* src = bf + (s + (dim ? M : 0)) * B2 + 4 * h;
      float* dst = sg + (dim ? S_BY : S_BX) + j * 16 + 8 * h;
      cp16(dst, src);
      cp16(dst + 4, src + 2);
    } break;
    case 6:
      cp8(sg + S_W + 4 * j, w + s);
      cp8(sg + S_W + 4 * j + 2, w + M + s);
      if (with_u) cp8(sg + S_U + 2 * j, u + ui);
      break;
    default:
      cp4(sg + S_FL + 2 * j, fl + s);
      cp4(sg + S_FL + 2 * j + 1, fl + M + s);
      break;
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// all but the most recent STAGES - 2 copy groups complete
__device__ __forceinline__ void cp_wait_stage() { asm volatile("cp.async.wait_group %0;\n" ::"n"(STAGES - 2) : "memory"); }
// the hi part of x at float offset oh, the lo part at ol
__device__ __forceinline__ void put2o(float* op, int oh, int ol, float x) {
  float hi, lo;
  split(x, hi, lo);
  op[oh] = hi;
  op[ol] = lo;
}
// float offset of row r (column part excluded): 8-row group and row within it
__device__ __forceinline__ int ro(int r) { return (r >> 3) * GRP + (r & 7) * 4; }

}  // namespace tc5

static __global__ void __launch_bounds__(160, 4) k_spread2d_tc5(
    const int32_t* __restrict__ work, const int32_t* __restrict__ order, const int32_t* __restrict__ fl,
    const float* __restrict__ win, const float2* __restrict__ w, const float2* __restrict__ bf,
    const float2* __restrict__ u, const int32_t* __restrict__ perm, int64_t M, int nbx, float2* __restrict__ part,
    int64_t stride, int* __restrict__ err) {
  using namespace tc5;
  extern __shared__ __align__(1024) float smt[];
  float* sm = smt;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + O_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + O_BAR + 2 * NBUF);
  volatile int* abort_s = reinterpret_cast<volatile int*>(sm + O_BAR + 2 * NBUF + 1);
  const int it = order[blockIdx.x];  // work item (larger items launch first)
  const int bin = work[3 * it], s0 = work[3 * it + 1], s1 = work[3 * it + 2];
  const int ox = (bin % nbx) * TILE, oy = (bin / nbx) * TILE;
  const int nbat = (s1 - s0 + SB - 1) / SB;
  if (nbat <= 0) {  // an empty item contributes a zero tile
    float4* out = reinterpret_cast<float4*>(part + it * stride);
    for (int i = tid; i < PART / 2; i += THREADS) out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // the caller-order index of this thread's sample in batch b (staging part PART_U only)
  const int ju = tid & (SB - 1);
  auto uindex = [&](int b) -> int {
    const int64_t s = s0 + (int64_t)b * SB + ju;
    if ((tid >> 4) != PART_U || b >= nbat || s >= s1) return 0;
    return perm ? perm[s] : (int)s;
  };
  // batches 0 .. STAGES-2 in flight before the loop (one copy group each)
#pragma unroll
  // (the sample values u may be written by the kernel before this one in the
  // stream: they are read only after griddepcontrol.wait below)
  for (int pb = 0; pb < STAGES - 1; ++pb) {
    if (pb < nbat && tid < BUILDERS)
      stage(sm + O_STAGE + pb * S_SIZE, tid, s0 + pb * SB, min(SB, s1 - s0 - pb * SB), win, w, bf, u, uindex(pb),
            fl, M, false);
    cp_commit();
  }
  int ui_next = (tid < BUILDERS) ? uindex(STAGES - 1) : 0;  // loaded one batch before it is staged
  {
    float4* z = reinterpret_cast<float4*>(sm);
    for (int i = tid; i < NBUF * BUF / 4; i += THREADS) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "n"(TM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NBUF; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar + i)));
    *abort_s = 0;
  }
  // Launched as a programmatic dependent of the interpolation in a CG step, the
  // CTA reaches this point while that kernel may still run: everything above
  // reads only the plan's tables.  Wait for the previous kernel's writes, then
  // stage the sample values of the first batches.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid < BUILDERS && (tid >> 4) == PART_U) {
#pragma unroll
    for (int pb = 0; pb < STAGES - 1; ++pb) {
      const int64_t s = s0 + (int64_t)pb * SB + (tid & (SB - 1));
      if (pb < nbat && s < s1)
        *reinterpret_cast<float2*>(sm + O_STAGE + pb * S_SIZE + S_U + 2 * (tid & (SB - 1))) = u[uindex(pb)];
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tb = *tslot;
  bool aborted = false;
  if (wid == 4) {  // the MMA warp: one lane issues both GEMMs of each batch once its operands are built
    for (int bt = 0; bt < nbat; ++bt) {
      const int q = bt % NBUF;
      nb_sync(1 + q, THREADS);
      if (*abort_s) break;
      if (lane == 0) {
        fence_after();
        const uint32_t base = saddr(sm + q * BUF);
#pragma unroll
        for (int t = 0; t < SB / 8; ++t) {
          const uint32_t acc = (bt > 0 || t > 0) ? 1u : 0u;
          mma_tf32(tb + TM_D1, sdesc(base + 4 * O_A1 + 256 * t), sdesc(base + 4 * O_B1 + 256 * t), ID1, acc);
          mma_tf32(tb + TM_D2, sdesc(base + 4 * O_A2 + 256 * t), sdesc(base + 4 * O_B2 + 256 * t), ID2, acc);
        }
        commit(bar + q);
      }
      __syncwarp();
    }
  } else {
  // build role: sample slot j of the batch, tap / boundary index a; offsets of the
  // slot's column and of the rows that do not move with the sample's position
  const int j = wid * 4 + (lane >> 3), a = lane & 7;
  const int cj = (j >> 2) * 32 + (j & 3);
  const int ra = ro(a) + cj;  // row a (< 8) of any operand, this column
  int pox_[NBUF], poy_[NBUF];  // the slot's window rows (offsets) in each buffer
#pragma unroll
  for (int i = 0; i < NBUF; ++i) pox_[i] = poy_[i] = -1;
  for (int bt = 0; bt < nbat; ++bt) {
    const int q = bt % NBUF;
    const int sb = s0 + bt * SB, nb = min(SB, s1 - sb);
    // the MMAs of batch bt - NBUF read buffer q (phase (bt / NBUF - 1) of its mbarrier)
    if (tid == 0 && bt >= NBUF && !wait_parity(bar + q, ((bt / NBUF) & 1) ^ 1)) *abort_s = 1;
    cp_wait_stage();
    nb_sync(NB_BUILD, BUILDERS);  // staging of batch bt visible; buffer q and staging buffer (bt-1) % STAGES free
    if (*abort_s) {
      aborted = true;
      nb_arrive(1 + q, THREADS);  // release the MMA warp, which then sees the abort
      break;
    }
    {
      const int nbt = bt + STAGES - 1;
      if (nbt < nbat)
        stage(sm + O_STAGE + (nbt % STAGES) * S_SIZE, tid, s0 + nbt * SB, min(SB, s1 - s0 - nbt * SB), win, w, bf, u,
              ui_next, fl, M);
      cp_commit();
      ui_next = uindex(nbt + 1);
    }
    float* ob = sm + q * BUF;
    const float* st = sm + O_STAGE + (bt % STAGES) * S_SIZE;
    int pox = -1, poy = -1;
#pragma unroll
    for (int i = 0; i < NBUF; ++i)
      if (i == q) pox = pox_[i], poy = poy_[i];
    if (pox >= 0) {  // clear the window entries of the slot's previous sample
      ob[O_A1 + pox] = 0.f;
      ob[O_A1 + pox + 3 * GRP] = 0.f;
      ob[O_A1 + pox + 8 * GRP] = 0.f;
      ob[O_A1 + pox + 11 * GRP] = 0.f;
      ob[O_B1 + poy] = 0.f;
      ob[O_B1 + poy + 3 * GRP] = 0.f;
      ob[O_B2 + pox] = 0.f;
      ob[O_B2 + pox + 5 * GRP] = 0.f;
    }
    __syncwarp();  // the slot's eight lanes are in this warp: clears before writes
    float2 us = make_float2(0.f, 0.f), wxs = us, wys = us, bxa = us, bya = us;
    float tx = 0.f, ty = 0.f;
    int px = 1, py = 1;  // empty slot: zero sample value and taps at a valid position
    if (j < nb) {
      const float4 ww = *reinterpret_cast<const float4*>(st + S_W + 4 * j);
      wxs = make_float2(ww.x, ww.y);
      wys = make_float2(ww.z, ww.w);
      us = *reinterpret_cast<const float2*>(st + S_U + 2 * j);
      const int* flj = reinterpret_cast<const int*>(st + S_FL + 2 * j);
      px = flj[0] - ox + 1;
      py = flj[1] - oy + 1;
      tx = st[S_WIN + j * 24 + a];
      ty = st[S_WIN + j * 24 + W + a];
      bxa = *reinterpret_cast<const float2*>(st + S_BX + j * 16 + 2 * a);
      bya = *reinterpret_cast<const float2*>(st + S_BY + j * 16 + 2 * a);
    }
    const int fx = ro(px + a) + cj, fy = ro(py + a) + cj;  // window row offsets (rows 24, 40, 64, 88 further
                                                           // are 3, 5, 8, 11 row groups on)
#pragma unroll
    for (int i = 0; i < NBUF; ++i)
      if (i == q) pox_[i] = fx, poy_[i] = fy;
    const float2 v = cmulc(cmulc(us, wxs), wys);
    const float2 v0 = cmulc(cmulc(us, wys), bxa);
    const float2 v1 = cmulc(cmulc(us, wxs), bya);
    const float2 ak = cmulc(us, bxa);
    float* A1 = ob + O_A1;
    float* B1 = ob + O_B1;
    float* A2 = ob + O_A2;
    float* B2o = ob + O_B2;
    put2o(A1, fx, fx + 8 * GRP, v.x * tx);                        // rows px+a, 64+px+a
    put2o(A1, fx + 3 * GRP, fx + 11 * GRP, v.y * tx);             // rows 24+px+a, 88+px+a
    put2o(A1, ra + 6 * GRP, ra + 14 * GRP, v0.x);                 // rows 48+a, 112+a
    put2o(A1, ra + 7 * GRP, ra + 15 * GRP, v0.y);                 // rows 56+a, 120+a
    put2o(B1, fy, fy + 3 * GRP, ty);                              // rows py+a, 24+py+a
    put2o(A2, ra, ra + 4 * GRP, v1.x);                            // rows a, 32+a
    put2o(A2, ra + GRP, ra + 5 * GRP, v1.y);                      // rows 8+a, 40+a
    put2o(A2, ra + 2 * GRP, ra + 6 * GRP, ak.x);                  // rows 16+a, 48+a
    put2o(A2, ra + 3 * GRP, ra + 7 * GRP, ak.y);                  // rows 24+a, 56+a
    put2o(B2o, fx, fx + 5 * GRP, tx);                             // rows px+a, 40+px+a
    put2o(B2o, ra + 3 * GRP, ra + 8 * GRP, bya.x);                // rows 24+a, 64+a
    put2o(B2o, ra + 4 * GRP, ra + 9 * GRP, -bya.y);               // rows 32+a, 72+a
    fence_async_smem();  // generic-proxy stores visible to the tensor core's reads
    nb_arrive(1 + q, THREADS);
  }
  }
  // all MMAs done: the last commit tracks every earlier MMA of the issuing thread
  const int last = nbat - 1;
  cp_wait_all();
  __syncthreads();  // every commit issued (or the loop left on an abort)
  if (tid == 0 && !*abort_s && !wait_parity(bar + last % NBUF, (last / NBUF) & 1)) *abort_s = 1;
  fence_before();
  __syncthreads();
  fence_after();
  if (*abort_s) {
    if (tid == 0) {
      atomicExch(err, 1);
      // the MMAs of the batches this CTA issued, once more with a bound, before TMEM is freed
      for (int bt = max(0, last - NBUF + 1); bt <= last; ++bt) wait_parity(bar + bt % NBUF, (bt / NBUF) & 1);
    }
    fence_before();
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "n"(TM_COLS));
    return;
  }
  float* H = sm + E_H;  // [64][LX]: hi*hi + hi*lo of D1 rows 0..63, columns 0..23
  float* X = sm + E_X;  // [64][LX]: lo*hi of D1 rows 64..127, columns 0..23
  float* Y = sm + E_Y;  // [32][LZ]: lo*hi of D2 rows 32..63, columns 0..39
  float* Z = sm + E_Z;  // [32][LZ]: hi*hi + hi*lo of D2 rows 0..31, columns 0..39
  const uint32_t lanes = (uint32_t)(32 * (wid & 3)) << 16;
  if (wid == 4) {
  } else if (wid >= 2) {
#pragma unroll
    for (int c = 0; c < 24; c += 8) {
      float v[8];
      tld8(tb + lanes + TM_D1 + c, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) X[(32 * (wid - 2) + lane) * LX + c + e] = v[e];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 24; c += 8) {
      float v[8], g[8];
      tld8(tb + lanes + TM_D1 + c, v);
      tld8(tb + lanes + TM_D1 + 24 + c, g);
#pragma unroll
      for (int e = 0; e < 8; ++e) H[(32 * wid + lane) * LX + c + e] = v[e] + g[e];
    }
#pragma unroll
    for (int c = 0; c < 40; c += 8) {
      float v[8], g[8];
      tld8(tb + lanes + TM_D2 + c, v);
      if (wid == 0) tld8(tb + lanes + TM_D2 + 40 + c, g);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (wid == 0) Z[lane * LZ + c + e] = v[e] + g[e];
        else Y[lane * LZ + c + e] = v[e];
      }
    }
  }
  fence_before();
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "n"(TM_COLS));
  // the partial tile in the layout of k_spread2d, consecutive threads on consecutive values
  float2* out = part + it * stride;
  for (int o = tid; o < PART; o += THREADS) {
    float re, im;
    if (o < PW * PW) {  // interior P[x][y]: D1 rows x (Re), 24 + x (Im)
      const int x = o / PW, y = o - x * PW;
      re = H[x * LX + y] + X[x * LX + y];
      im = H[(24 + x) * LX + y] + X[(24 + x) * LX + y];
    } else if (o < PW * PW + B2 * PW) {  // x-sides S0[k][y]: D1 rows 48 + k, 56 + k
      const int t = o - PW * PW, k = t / PW, y = t - k * PW;
      re = H[(48 + k) * LX + y] + X[(48 + k) * LX + y];
      im = H[(56 + k) * LX + y] + X[(56 + k) * LX + y];
    } else if (o < PW * PW + 2 * B2 * PW) {  // y-sides S1[k][x]: D2 rows k, 8 + k
      const int t = o - PW * PW - B2 * PW, k = t / PW, x = t - k * PW;
      re = Z[k * LZ + x] + Y[k * LZ + x];
      im = Z[(8 + k) * LZ + x] + Y[(8 + k) * LZ + x];
    } else {  // corners: A (D2 rows 16 + kx, 24 + kx) times conj(by) (columns 24 + ky, 32 + ky)
      const int t = o - PW * PW - 2 * B2 * PW, kx = t % B2, ky = t / B2;
      const float rr = Z[(16 + kx) * LZ + 24 + ky] + Y[(16 + kx) * LZ + 24 + ky];
      const float ir = Z[(24 + kx) * LZ + 24 + ky] + Y[(24 + kx) * LZ + 24 + ky];
      const float ri = Z[(16 + kx) * LZ + 32 + ky] + Y[(16 + kx) * LZ + 32 + ky];
      const float ii = Z[(24 + kx) * LZ + 32 + ky] + Y[(24 + kx) * LZ + 32 + ky];
      re = rr - ii;
      im = ri + ir;
    }
    out[o] = make_float2(re, im);
  }
  // the reductions launched as this kernel's programmatic dependent may start
  // once every CTA has written its partial tile (they wait for the grid anyway)
  asm volatile("griddepcontrol.launch_dependents;");
}

}  // namespace dev
}  // namespace gs

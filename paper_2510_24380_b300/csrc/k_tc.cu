// k_tc.cu -- 16-bit tensor-core enumeration kernel for sm_103a (tcgen05 + TMEM + bulk TMA),
// instantiated for BF16 and FP16 operands (one format for tables, activations and weights).
//
// Head shape: d -> 256 -> 256 -> n_out (n_out <= 16), activation after layers 1 and 2.
// Per tile of 128 compounds (rows): inner block b (rows q0 + [0, 128) of the reaction's inner
// slots) x one outer index o; each CTA walks an equal contiguous share of the launch's tiles:
//   layer 1, structure-exploiting form (Eq. apex generalized to W_1): z_1 = R(row) + p(o), where
//     R(row) = sum of the row's inner-slot P rows (resident in the producer's registers for the
//     whole item) and p(o) = the outer slot's P row (one broadcast load per tile);
//     a_1 = act(z_1) -> 16-bit -> shared memory in the UMMA SW128 K-major layout;
//   layer 2: D2[128 x 256] = a_1 W_2^T, tcgen05.mma (A, B from shared memory), FP32 in TMEM;
//   epilogue 1: a_2 = act(D2 + b_2) -> 16-bit pairs packed back into the same TMEM columns;
//   layer 3: D3[128 x 16] = a_2 W_3^T, tcgen05.mma with A read from TMEM;
//   epilogue 2: outputs -> queries (objective, boxes, admission) or a raw dump.
// SiLU is evaluated as h + h tanh(h) with h = z/2, on packed 16-bit pairs (add / tanh.approx /
// fma .bf16x2 or .f16x2: 1.5 issue slots and one MUFU element per activation); the 1/2 is folded into P
// (layer 1) and into the W_2 image and b_2 (layer 2), all exact in binary. In a BF16 pass 3/8 of the
// layer-2 activations take an ex2 form instead (silu2_ex2_bf16: half the MUFU time, five more FMA-pipe
// instructions), which moves part of the MUFU load, the kernel's bound, to the FMA pipe.
//
// Warp roles (736 threads, one CTA per SM):
//   warps 0-3   query warps: D3 of each tile -> outputs -> queries (warp w reads TMEM lanes 32w..)
//   warps 4-19  math warps, thread (g, m) = K quarter g, tile row m: per step, layer 1 of the
//               next tile (stage g of a_1) and then the layer-2 activation of the previous tile
//               (accumulator columns [64g, 64g + 64), rows of its TMEM lane quarter)
//   warp 20     TMEM allocation; lane 0 issues the layer-2 MMAs and their commits
//   warp 21     lane 0 bulk-copies (TMA) each tile's outer synthon row into a 4-slot ring
//   warp 22     lane 0 issues each tile's layer-3 MMAs once its a_2 is complete
// TMEM: 512 columns = two 256-column accumulators (double buffer); a_2 of quarter g overwrites
// columns [64g, 64g + 32) of its buffer, the four layer-3 partial sums use [32, 64) and [96, 128).
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel records
// APX_ERR_TIMEOUT in the status word, every role leaves its loop, and TMEM is released.
#include <algorithm>
#include <cstring>
#include "common.cuh"
#include "tc_sync.cuh"

#define TC_EPI_WARPS 4
#define TC_PROD_WARPS 16
#define TC_MMA_WARP (TC_EPI_WARPS + TC_PROD_WARPS)
#define TC_LOAD_WARP (TC_MMA_WARP + 1)
#define TC_L3_WARP (TC_LOAD_WARP + 1)
#define TC_THREADS ((TC_L3_WARP + 1) * 32)
#define TC_OROW_SLOTS 4
// Layer 3 accumulates in four independent chains (K blocks c, c + 4, c + 8, c + 12 go to chain c),
// so that consecutive MMAs do not wait on each other; chain c uses 16 of the columns that layer
// 2's activation has freed, the upper half of quarter c / 2 of the 256-column buffer.
#define TC_L3_CHAINS 4
__host__ __device__ constexpr uint32_t tc_d3_col(int c) { return 64u * (uint32_t)(c >> 1) + 32u + 16u * (uint32_t)(c & 1); }

// Query parameters cached in shared memory for the whole launch (one entry per query slot). The
// boxes are stored per output (several constraints on one output intersect; +-inf where an output
// is unconstrained) as FP16 pairs, element j of pair j / 2 for output j, so that the epilogue tests
// two outputs per packed instruction with no branch per output. Bounds are rounded so that the
// FP16 tests never err the wrong way (tc_box_admit / tc_box_sure): the admission box outward, the
// sure box inward and one more FP16 step inward.
struct SlotParams {
  float w[APEX_MAX_OBJECTIVES];  // zero beyond n_obj
  uint32_t lo_w[8], hi_w[8];     // admission box (widened by the pass margin)
  uint32_t lo_s[8], hi_s[8];     // "sure" box (shrunk by the margin)
  float admit;
  unsigned cmask;
  int n_obj;
  unsigned cap;          // candidate buffer of the query (copied from its slot: no global loads
  float *keys;           // on the append path)
  long long *ids;
};

// Shared-memory map (offsets from a 1024-byte aligned base), per operand format FMT (0 = BF16,
// 1 = FP16, 2 = FP8 e4m3 for layer 2, FP16 for layer 3). 16-bit: W_2 128 KB, W_3 8 KB, a_1 as four
// K-quarter stages of 16 KB (one tile). FP8: W_2 64 KB, W_3 8 KB (FP16), a_1 double-buffered: two
// tiles x two K-halves of 16 KB (128 K elements per 128-byte row), plus the per-channel
// dequantization scales of W_2.
#define TC_NBAR 35
template <int FMT>
struct TcL {
  static constexpr bool F8 = FMT == 2;
  static constexpr uint32_t W2 = 0u, W2_BYTES = F8 ? 65536u : 131072u;
  static constexpr uint32_t W3 = W2 + W2_BYTES, W3_BYTES = 8192u;
  static constexpr uint32_t A1 = W3 + W3_BYTES, STAGE = 16384u;
  static constexpr uint32_t OROW = A1 + 4u * STAGE;             // outer-row ring: 4 x 512 B (16-bit x 256)
  static constexpr uint32_t B2 = OROW + TC_OROW_SLOTS * 512u;   // 16-bit: 128 packed pairs; FP8: 256 floats
  static constexpr uint32_t S2 = B2 + 1024u;                     // FP8: 256 per-channel scales
  static constexpr uint32_t B3 = S2 + (F8 ? 1024u : 0u);         // 16 floats
  static constexpr uint32_t QP = B3 + 64u;                       // APEX_MAX_ACTIVE x SlotParams
  static constexpr uint32_t BAR = QP + (uint32_t)(APEX_MAX_ACTIVE * sizeof(SlotParams));
  static constexpr uint32_t MISC = BAR + 8u * TC_NBAR;
  static constexpr uint32_t QLIST = MISC + 64u;                  // per query warp: its run's query slots
  static constexpr uint32_t RING = (QLIST + 4u * APEX_MAX_ACTIVE + 15u) & ~15u;  // 4 tail-pool ranges {a, b}
  static constexpr uint32_t SMEM = RING + 64u + 1024u;            // + alignment slack
};
static_assert(sizeof(SlotParams) == 224, "SlotParams layout");
static_assert(TcL<0>::SMEM <= 232448 && TcL<1>::SMEM <= 232448 && TcL<2>::SMEM <= 232448, "shared memory budget");
static_assert(TcL<0>::A1 % 1024 == 0 && TcL<2>::A1 % 1024 == 0 && TcL<0>::QP % 16 == 0 && TcL<2>::QP % 16 == 0,
              "alignment");

// barrier indices
#define B_FULL(s) (s)
#define B_EMPTY(s) (4 + (s))
#define B_D2FULL(b) (8 + (b))
#define B_D2EMPTY(b) (10 + (b))
#define B_A2FULL(b) (12 + (b))
#define B_D3FULL(b) (14 + (b))
#define B_W 16
#define B_DRAIN 17
#define B_DRAIN3 26  // layer-3 issuer's drain
#define B_OFULL(r) (18 + (r))
#define B_OEMPTY(r) (22 + (r))
#define B_RFULL(e) (27 + (e))   // tail-pool range ring (entry e of 4): published by the loader
#define B_REMPTY(e) (31 + (e))  // ... released by every other warp role (TC_RING_READERS arrivals)
#define TC_RING_READERS (TC_PROD_WARPS + TC_EPI_WARPS + 2)

// UMMA shared-memory descriptor: SW128 K-major, 8-row atoms 1024 B apart (SBO)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}
// instruction descriptor: kind::f16, A and B of the same 16-bit type (FMT 0 = BF16 -> format
// code 1, FMT 1 = F16 -> format code 0), FP32 accumulator, both K-major
__host__ __device__ constexpr uint32_t idesc_16(int M, int N, int FMT) {
  return (1u << 4) | ((FMT == 0 ? 1u : 0u) << 7) | ((FMT == 0 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor: kind::f8f6f4, E4M3 x E4M3 (format code 0) -> FP32, both K-major
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}
// kind::f8f6f4 (8-bit operands) forms
__device__ __forceinline__ void mma_ss_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,"
      "%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// wait::ld that also ties the loaded registers to the wait, so no use of them is scheduled
// before it
__device__ __forceinline__ void tmem_wait_ld_dep(uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]), "+r"(v[8]),
        "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]),
        "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]),
        "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
      :
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld_dep16(uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]), "+r"(v[8]),
        "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
      :
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// activation of a value already in the activation's input space (h = z/2 for SiLU)
template <int ACT>
__device__ __forceinline__ float act_h(float h) {
  if (ACT == APEX_ACT_SILU) return fmaf(h, tanh_fast(h), h);
  if (ACT == APEX_ACT_RELU) return fmaxf(h, 0.f);
  return h;
}
// Packed 16-bit math, 2 elements per instruction (issue slots, not MUFU rate, bound this path).
// FMT 0 = BF16 (8 mantissa bits), FMT 1 = FP16 (11 mantissa bits, same instruction rates).
#define APX_PK2(NAME, OP)                                                 \
  template <int FMT>                                                      \
  __device__ __forceinline__ uint32_t NAME(uint32_t a, uint32_t b) {      \
    uint32_t d;                                                           \
    if (FMT == 0)                                                         \
      asm(OP ".bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));           \
    else                                                                  \
      asm(OP ".f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));            \
    return d;                                                             \
  }
APX_PK2(add2, "add.rn")
APX_PK2(max2, "max")
#undef APX_PK2
template <int FMT>
__device__ __forceinline__ uint32_t tanh2(uint32_t a) {
  uint32_t d;
  if (FMT == 0)
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(d) : "r"(a));
  else
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}
template <int FMT>
__device__ __forceinline__ uint32_t fma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  if (FMT == 0)
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  else
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// activation of a packed pair already in the activation's input space (h = z/2 for SiLU):
// SiLU(2h) = h + h tanh(h)
template <int ACT, int FMT>
__device__ __forceinline__ uint32_t act2(uint32_t h) {
  if (ACT == APEX_ACT_SILU) return fma2<FMT>(h, tanh2<FMT>(h), h);
  if (ACT == APEX_ACT_RELU) return max2<FMT>(h, 0u);
  return h;
}
// SiLU(2h) of a packed BF16 pair through the MUFU's ex2, which costs half its tanh:
// h + |h| tanh|h|, tanh|h| = (1 - e) / (1 + e), e = exp(-2|h|) = 2^(-K|h|) with K = 2 log2(e)
// rounded to BF16 (2.890625). (1 - e) / (1 + e) is P(e) = 1 + c1 e + c2 e^2 + c3 e^3 on the FMA
// pipe: a least-squares fit over e in (0, 1] weighted by |h| (the weight of its error in the
// activation), reweighted towards equal ripple, P(0) = 1 held (exact for large |h|), each
// coefficient rounded to BF16 and the others refitted around it, with the rounding of K folded
// into the target. Evaluated in BF16 its error stays at the level of the result's own rounding:
// over h in [-9, 9], mean |error| 1.84e-3 against 1.77e-3 for the tanh.approx form, the same
// maximum. The sign of h goes into P by one logic operation (h + h sign(h) P).
__device__ __forceinline__ uint32_t silu2_ex2_bf16(uint32_t h) {
  constexpr uint32_t SIGN = 0x80008000u;
  const uint32_t u = fma2<0>(h, 0x40394039u, SIGN) | SIGN;  // -K|h| (K h + (-0), sign set)
  uint32_t e;
  asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(e) : "r"(u));
  uint32_t p = fma2<0>(0xbf41bf41u, e, 0x3fd83fd8u);  // c3 = -0.75390625, c2 = 1.6875
  p = fma2<0>(p, e, 0xbffebffeu);                     // c1 = -1.984375
  p = fma2<0>(p, e, 0x3f803f80u);                     // 1
  return fma2<0>(h, p ^ (h & SIGN), h);
}
// Layer-2 activations of a BF16 pass that take silu2_ex2_bf16 instead of tanh.approx: pairs 2, 3
// and 7 of every 8 (3/8). The ex2 form takes five more FMA-pipe instructions per pair, so moving a
// share of the pairs relieves the MUFU only until issue slots bind; this share measured fastest
// (1/8 to 1/2 of layer 2 and 1/8 to 1/2 of layer 1 were timed; layer 1 gained less).
#define TC_EX2_PAIRS 0x8Cu
// two floats -> packed 16-bit pair (round to nearest even), lo in bits [0, 16)
template <int FMT>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t w;
  if (FMT == 0)
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  return w;
}
// two packed f16 pairs (elements k, k+1 and k+2, k+3) -> four e4m3 bytes, element k in the low
// byte (round to nearest even, saturating at +-448)
__device__ __forceinline__ uint32_t e4m3x4(uint32_t h01, uint32_t h23) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(lo) : "r"(h01));
  asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(hi) : "r"(h23));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}
// packed 16-bit pair -> the two floats (exact)
template <int FMT>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  if (FMT == 0) return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  float lo, hi;
  asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n cvt.f32.f16 %0, l;\n cvt.f32.f16 %1, h;\n}" : "=f"(lo), "=f"(hi) : "r"(w));
  return make_float2(lo, hi);
}

// FP16 bound rounding (bit level; x is never NaN): the largest FP16 value <= x, the smallest >= x,
// and one FP16 step down / up.
__device__ __forceinline__ uint16_t f16_rn(float x) {
  uint16_t h;
  asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
  return h;
}
__device__ __forceinline__ float f16_val(uint16_t h) {
  float x;
  asm("cvt.f32.f16 %0, %1;" : "=f"(x) : "h"(h));
  return x;
}
__device__ __forceinline__ uint16_t f16_down(uint16_t h) {  // next FP16 value below (-inf stays)
  if (h == 0x0000u) return 0x8001u;
  if (h == 0xfc00u) return h;
  return (h & 0x8000u) ? (uint16_t)(h + 1u) : (uint16_t)(h - 1u);
}
__device__ __forceinline__ uint16_t f16_up(uint16_t h) {  // next FP16 value above (+inf stays)
  if (h == 0x8000u) return 0x0001u;
  if (h == 0x7c00u) return h;
  return (h & 0x8000u) ? (uint16_t)(h - 1u) : (uint16_t)(h + 1u);
}
__device__ __forceinline__ uint16_t f16_rd(float x) {
  const uint16_t h = f16_rn(x);
  return f16_val(h) > x ? f16_down(h) : h;
}
__device__ __forceinline__ uint16_t f16_ru(float x) {
  const uint16_t h = f16_rn(x);
  return f16_val(h) < x ? f16_up(h) : h;
}
// The row's 16 outputs as FP16 pairs (round to nearest, saturated to the finite range: both are
// monotonic, so an output inside a box stays inside its outward-rounded FP16 image)
__device__ __forceinline__ void tc_outputs_f16(const float (&o)[16], uint32_t (&h)[8]) {
#pragma unroll
  for (int n = 0; n < 8; ++n) asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(h[n]) : "f"(o[2 * n + 1]), "f"(o[2 * n]));
}
// Box tests on FP16 pairs: inside iff every o - lo and hi - o is >= 0, i.e. has a clear sign bit
// (the difference of two FP16 values is zero only when they are equal, and then +0). Admission box
// [rd(lo), ru(hi)]: every output inside [lo, hi] passes (extra passes near the bounds only add
// candidates). Sure box [up(ru(lo)), down(rd(hi))]: an FP16 image at or above up(ru(lo)) comes from
// an output above ru(lo) >= lo, so every output that passes is inside [lo, hi].
__device__ __forceinline__ bool tc_box(const uint32_t (&h)[8], const uint32_t *lo, const uint32_t *hi) {
  uint32_t neg = 0u;
#pragma unroll
  for (int n = 0; n < 8; n += 4) {
    const uint4 l = *reinterpret_cast<const uint4 *>(lo + n), u = *reinterpret_cast<const uint4 *>(hi + n);
    const uint32_t lv[4] = {l.x, l.y, l.z, l.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t a, b;
      asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(a) : "r"(h[n + e]), "r"(lv[e]));
      asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(b) : "r"(uv[e]), "r"(h[n + e]));
      neg |= a | b;
    }
  }
  return (neg & 0x80008000u) == 0u;
}

// Sec. 3 / Eq. apex_topk per compound (one row per lane, all 32 lanes call it): objective,
// admission threshold, widened box (admission) and shrunk box ("sure"), then a warp-aggregated
// append to the query's candidate buffer in global memory. Parameters come from shared memory.
__device__ __forceinline__ void tc_apply_query_box(const SlotParams &P, QuerySlot *Q, bool pass, float f, long long id,
                                                   const uint32_t (&h)[8]) {
  pass = pass && tc_box(h, P.lo_w, P.hi_w);
  if (__ballot_sync(0xffffffffu, pass) == 0u) return;  // no lane inside the widened boxes
  const bool sure = tc_box(h, P.lo_s, P.hi_s);
  const unsigned pos = apx_warp_reserve(&Q->count, pass);
  if (pass) {
    if (pos < P.cap) {
      P.keys[pos] = f;
      P.ids[pos] = id | (sure ? 0LL : APX_UNSURE_BIT);
    } else {
      apx_note_dropped(Q, f);
    }
  }
}
__device__ __forceinline__ void tc_apply_query_slow(const SlotParams &P, QuerySlot *Q, bool pass, float f, long long id,
                                                    const float (&o)[16]) {
  uint32_t h[8];  // the row's outputs as FP16 pairs (formed per test: cheaper than keeping them live)
  tc_outputs_f16(o, h);
  tc_apply_query_box(P, Q, pass, f, id, h);
}

// objective of one query: its weights are zero beyond n_obj, so a fixed-length dot product serves
template <int NW>
__device__ __forceinline__ float tc_objective(const SlotParams &P, const float (&o)[16]) {
  float f0 = 0.f, f1 = 0.f;  // two independent partial sums
#pragma unroll
  for (int j = 0; j < NW; j += 4) {
    const float4 w = *reinterpret_cast<const float4 *>(&P.w[j]);
    f0 = fmaf(w.x, o[j], f0);
    f1 = fmaf(w.y, o[j + 1], f1);
    f0 = fmaf(w.z, o[j + 2], f0);
    f1 = fmaf(w.w, o[j + 3], f1);
  }
  return f0 + f1;
}

// Sec. 3 / Eq. apex_topk per compound (one row per lane, all 32 lanes call it): objective,
// admission threshold, widened box (admission) and shrunk box ("sure"), then a warp-aggregated
// append to the query's candidate buffer in global memory. Parameters come from shared memory.
// Objectives are formed for TC_QGROUP queries at a time (independent dot products); the constraint
// boxes are read only for the queries that some lane of the warp admits on the objective. The
// query slots of the run come as a list in shared memory (built once per run), so the per-tile
// loop uses no bit scans (those would queue on the MUFU pipe behind the activations).
#define TC_QGROUP 2  // queries per step of the epilogue loop (wider groups spill registers)
template <int NW>
__device__ __forceinline__ void tc_apply_queries_n(const SlotParams *qp, QuerySlot *slots, const unsigned char *qlist,
                                                   int nq, bool valid, long long id, const float (&o)[16]) {
  uint32_t h[8];  // the row's outputs as FP16 pairs, formed once for every query's box tests
  tc_outputs_f16(o, h);
  for (int i = 0; i < nq; i += TC_QGROUP) {
    int sq[TC_QGROUP];
#pragma unroll
    for (int u = 0; u < TC_QGROUP; ++u) sq[u] = i + u < nq ? (int)qlist[i + u] : -1;
    float f[TC_QGROUP];
    bool pass[TC_QGROUP];
#pragma unroll
    for (int u = 0; u < TC_QGROUP; ++u) {
      const SlotParams &P = qp[sq[u] < 0 ? 0 : sq[u]];
      f[u] = tc_objective<NW>(P, o);
      pass[u] = valid && sq[u] >= 0 && f[u] >= P.admit;
    }
#pragma unroll
    for (int u = 0; u < TC_QGROUP; ++u)
      if (__ballot_sync(0xffffffffu, pass[u]) != 0u) tc_apply_query_box(qp[sq[u]], slots + sq[u], pass[u], f[u], id, h);
  }
}

// Launches with at most TC_FEWQ queries: every objective first (branch-free, one admission bit
// per query), one warp reduction, then the append path for the queries some lane admits. The
// kernel is instantiated separately for this form, so its registers do not depend on the
// many-query form's.
#define TC_FEWQ 2
template <int NW>
__device__ __forceinline__ void tc_apply_queries_few(const SlotParams *qp, QuerySlot *slots, const unsigned char *qlist,
                                                     int nq, bool valid, long long id, const float (&o)[16]) {
  unsigned bits = 0u;
  if (valid) {
    for (int i = 0; i < nq; ++i) {
      const SlotParams &P = qp[qlist[i]];
      bits |= (unsigned)(tc_objective<NW>(P, o) >= P.admit) << i;
    }
  }
  const unsigned any = __reduce_or_sync(0xffffffffu, bits);
  for (int i = 0; i < nq; ++i)
    if ((any >> i) & 1u) {  // warp-uniform
      const int sq = qlist[i];
      const SlotParams &P = qp[sq];
      tc_apply_query_slow(P, slots + sq, ((bits >> i) & 1u) != 0u, tc_objective<NW>(P, o), id, o);
    }
}

template <bool FEWQ>
__device__ __forceinline__ void tc_apply_queries(const SlotParams *qp, QuerySlot *slots, const unsigned char *qlist,
                                                 int nq, bool valid, long long id, const float (&o)[16], int n_obj) {
  if (FEWQ) {
    if (n_obj <= 8)
      tc_apply_queries_few<8>(qp, slots, qlist, nq, valid, id, o);
    else
      tc_apply_queries_few<16>(qp, slots, qlist, nq, valid, id, o);
  } else {
    if (n_obj <= 8)
      tc_apply_queries_n<8>(qp, slots, qlist, nq, valid, id, o);
    else
      tc_apply_queries_n<16>(qp, slots, qlist, nq, valid, id, o);
  }
}

// IDS: the rows of the launch are a list of compound ids (L.dump_ids[0, L.dump_n)), 128 per tile,
// each row summing the P rows of all its slots; the FP32 outputs go to L.dump (the start-
// threshold sample of a query). Otherwise the tiles come from the launch plan.
template <int ACT, int FMT, bool FEWQ, bool IDS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_head(const __grid_constant__ LaunchPlan L, const __grid_constant__ DevTables T, QuerySlot *slots, int *err) {
  using LY = TcL<FMT>;
  constexpr bool F8 = LY::F8;
  constexpr int PF = F8 ? 1 : FMT;  // 16-bit format of the table and the activation arithmetic (FP8: FP16)
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(sm);
  float *b2s = reinterpret_cast<float *>(sm + LY::B2);
  float *s2s = reinterpret_cast<float *>(sm + LY::S2);
  float *b3s = reinterpret_cast<float *>(sm + LY::B3);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + LY::MISC);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + LY::MISC + 8);
  auto bar = [&](int i) { return sbase + LY::BAR + 8u * (uint32_t)i; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // id lists: the list's length (read from the device when the launch gives it there) and its tiles
  const long long n_ids = IDS ? (L.dump_n_dev ? min(L.dump_n, (long long)*L.dump_n_dev) : L.dump_n) : 0;
  const long long launch_tiles = IDS ? (n_ids + APX_TILE - 1) / APX_TILE : L.total_tiles;
  // this CTA's share of the launch: tiles [t_begin, t_end), from the launch plan's cost-weighted
  // ranges when it has them (a tile that starts a run of tiles costs more), else equal counts;
  // walked by every role in the same order of runs
  const long long t_begin = L.cta_n == (int)gridDim.x ? L.cta_first[blockIdx.x]
                                                      : (long long)blockIdx.x * launch_tiles / gridDim.x;
  const long long t_end = L.cta_n == (int)gridDim.x ? L.cta_first[blockIdx.x + 1]
                                                    : (long long)(blockIdx.x + 1) * launch_tiles / gridDim.x;
  // Tail pool (L.pool_ctr != nullptr): after its own range a CTA takes chunks of the tiles past every
  // CTA's range, claimed by the loader warp and passed to the other roles through a 4-entry ring of
  // ranges in shared memory (a = -1: no more). Every role walks the same sequence of ranges.
  auto pool_next = [&](unsigned &n, long long &a, long long &b, bool whole_warp) -> bool {
    const int e = (int)(n & 3u);
    bool got = mbar_wait(bar(B_RFULL(e)), (n >> 2) & 1u, abort_flag, err);
    if (whole_warp) got = __all_sync(0xffffffffu, got);  // every lane gets here: no divergent exit
    if (!got) return false;
    const volatile long long *ring = reinterpret_cast<const volatile long long *>(sm + LY::RING) + 2 * e;
    a = ring[0];
    b = ring[1];
    if (whole_warp) __syncwarp();
    if (!whole_warp || lane == 0) mbar_arrive(bar(B_REMPTY(e)));
    ++n;
    return a >= 0;
  };
  auto pool_publish = [&](unsigned &n, long long a, long long b) -> bool {
    const int e = (int)(n & 3u);
    if (!mbar_wait(bar(B_REMPTY(e)), ((n >> 2) & 1u) ^ 1u, abort_flag, err)) return false;
    volatile long long *ring = reinterpret_cast<volatile long long *>(sm + LY::RING) + 2 * e;
    ring[0] = a;
    ring[1] = b;
    mbar_arrive(bar(B_RFULL(e)));
    ++n;
    return true;
  };
  if (tid == 0) {
    for (int s = 0; s < 4; ++s) {  // FP8: a K-half stage is written by the warps of two K quarters
      mbar_init(bar(B_FULL(s)), F8 ? 8 : 4);
      mbar_init(bar(B_EMPTY(s)), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_D2FULL(b)), 1);
      mbar_init(bar(B_D2EMPTY(b)), TC_EPI_WARPS);
      mbar_init(bar(B_A2FULL(b)), TC_PROD_WARPS);
      mbar_init(bar(B_D3FULL(b)), 1);
    }
    mbar_init(bar(B_W), 1);
    mbar_init(bar(B_DRAIN), 1);
    mbar_init(bar(B_DRAIN3), 1);
    for (int r = 0; r < TC_OROW_SLOTS; ++r) {
      mbar_init(bar(B_OFULL(r)), 1);
      mbar_init(bar(B_OEMPTY(r)), TC_PROD_WARPS);  // every math warp reads every outer row
    }
    for (int e = 0; e < 4; ++e) {
      mbar_init(bar(B_RFULL(e)), 1);
      mbar_init(bar(B_REMPTY(e)), TC_RING_READERS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    // W_2 (16 KB pieces) and W_3 images -> shared memory by bulk TMA
    mbar_expect_tx(bar(B_W), LY::W2_BYTES + LY::W3_BYTES);
    for (uint32_t off = 0; off < LY::W2_BYTES; off += 16384u)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              sbase + LY::W2 + off),
          "l"(T.w2img[FMT] + off), "r"(16384u), "r"(bar(B_W))
          : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sbase + LY::W3),
        "l"(T.w3img[PF]), "r"(LY::W3_BYTES), "r"(bar(B_W))
        : "memory");
  }
  if (!F8) {  // b_2 as packed 16-bit pairs: added to the packed accumulator pair in the activation
    for (int i = tid; i < 128; i += TC_THREADS)
      reinterpret_cast<uint32_t *>(b2s)[i] = pack2<PF>(T.b2s[2 * i], T.b2s[2 * i + 1]);
  } else {    // FP8: h = D * s_2[n] + b_2[n] in FP32 (per-channel dequantization of W_2)
    for (int i = tid; i < 256; i += TC_THREADS) {
      b2s[i] = T.b2s[i];
      s2s[i] = T.s2[i];
    }
  }
  for (int i = tid; i < 16; i += TC_THREADS) b3s[i] = T.b3[i];
  SlotParams *qp = reinterpret_cast<SlotParams *>(sm + LY::QP);
  if (L.mode == 0 && slots) {
    for (int s = warp; s < APEX_MAX_ACTIVE; s += TC_THREADS / 32) {
      if (!((L.qmask_all >> s) & 1ull)) continue;
      const QuerySlot *Q = slots + s;
      SlotParams &P = qp[s];
      if (lane < APEX_MAX_OBJECTIVES) P.w[lane] = Q->w[lane];
      if (lane < 16) {  // output `lane`: the intersection of the boxes of every constraint on it
        float lw = -INFINITY, hw = INFINITY, ls = -INFINITY, hs = INFINITY;
        bool any = false;
        for (int c = 0; c < Q->n_cons; ++c)
          if (Q->cons_idx[c] == lane) {
            any = true;
            lw = fmaxf(lw, Q->lo_w[c]);
            hw = fminf(hw, Q->hi_w[c]);
            ls = fmaxf(ls, Q->lo_s[c]);
            hs = fminf(hs, Q->hi_s[c]);
          }
        // FP16 images: admission box outward, sure box inward and one step further in (an infinite
        // bound stays infinite)
        const uint32_t b_lw = f16_rd(lw), b_hw = f16_ru(hw);
        const uint32_t b_ls = ls == -INFINITY ? 0xfc00u : f16_up(f16_ru(ls));
        const uint32_t b_hs = hs == INFINITY ? 0x7c00u : f16_down(f16_rd(hs));
        const uint32_t p_lw = b_lw | (__shfl_down_sync(0x0000ffffu, b_lw, 1) << 16);
        const uint32_t p_hw = b_hw | (__shfl_down_sync(0x0000ffffu, b_hw, 1) << 16);
        const uint32_t p_ls = b_ls | (__shfl_down_sync(0x0000ffffu, b_ls, 1) << 16);
        const uint32_t p_hs = b_hs | (__shfl_down_sync(0x0000ffffu, b_hs, 1) << 16);
        if ((lane & 1) == 0) {
          P.lo_w[lane >> 1] = p_lw;
          P.hi_w[lane >> 1] = p_hw;
          P.lo_s[lane >> 1] = p_ls;
          P.hi_s[lane >> 1] = p_hs;
        }
        const unsigned cm = __ballot_sync(0x0000ffffu, any);
        if (lane == 0) P.cmask = cm;
      }
      if (lane == 0) {
        P.admit = Q->admit;
        P.n_obj = Q->n_obj;
        P.cap = Q->cap;
        P.keys = Q->keys;
        P.ids = Q->ids;
      }
    }
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp >= TC_EPI_WARPS && warp < TC_MMA_WARP) {
    // ------------------------------------------------------------ math warps
    // Thread (g, m): tile row m (= TMEM lane; warp % 4 is the row quarter) and K quarter g
    // (64 columns = one a_1 stage). Step s: produce stage g of a_1 for tile s (layer 1), then
    // activate layer 2 of tile s - 1 on accumulator columns [64g, 64g + 64), writing a_2 back in
    // place. Producing first lets layer 2 of tile s run on the tensor pipe while layer 2 of tile
    // s - 1 is activated.
    const int p = tid - TC_EPI_WARPS * 32;
    const int g = p >> 7, m = p & 127;
    // FP8: a_1 times its power-of-two activation scale (exact in FP16) before the e4m3 conversion
    const uint32_t a1s = F8 ? pack2<1>(T.a1_inv, T.a1_inv) : 0u;
    const uint32_t row_off = (uint32_t)(m >> 3) * 1024u + (uint32_t)(m & 7) * 128u;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t R[32];  // resident inner sum of the producing item (64 columns), packed bf16 pairs
    long long tile = t_begin, rend = t_end;  // current range of tiles
    unsigned n_ring = 0;                       // tail-pool ranges read so far
    int left = 0;            // tiles left in the current run
    bool more = tile < rend;
    while (!more && L.pool_ctr && pool_next(n_ring, tile, rend, true)) more = tile < rend;
    bool need_r = more;
    bool ok = true;
    for (unsigned s = 0; ok; ++s) {
      const bool produce = more;
      if (produce) {
        if (need_r) {
          // the row's synthon of every summed slot (mixed radix, last slot fastest); unrolled over
          // the slot count so that the row pointers stay in registers
          const unsigned short *src[APEX_MAX_SLOTS];
          int ni = 0;
          bool row_ok;
          if constexpr (IDS) {  // every slot of the listed compound; each tile is its own run
            left = 1;
            const long long i = tile * APX_TILE + m;
            row_ok = i < n_ids;
            const long long id = row_ok ? (L.dump_ids[i] & APX_ID_MASK) : 0;
            int lo = 0, hi = T.n_rx - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
            }
            const RxnPlan *rp = T.rx + lo;
            long long rem = id - rp->id_first;
            ni = row_ok ? rp->n_slots : 0;
#pragma unroll
            for (int sl = APEX_MAX_SLOTS - 1; sl >= 0; --sl) {
              src[sl] = T.P16[PF] + g * 64;
              if (sl < ni) {
                const long long sz = rp->slot_size[sl];
                long long dig;
                rem = apx_divmod(rem, sz, &dig);
                src[sl] += (rp->slot_row[sl] + dig) * 256;
              }
            }
          } else {  // the inner slots of the tile's work item
            const TileRun I = apx_tile_run(L, T.rx, tile, rend);
            const RxnPlan *rp = I.rp;
            left = (int)(I.o_end - I.o_begin);
            const long long q = I.q0 + m;
            row_ok = q < rp->n_inner;
            long long rem = q;
            ni = row_ok ? rp->n_inner_slots : 0;
#pragma unroll
            for (int sl = APEX_MAX_SLOTS - 1; sl >= 0; --sl) {
              src[sl] = T.P16[PF] + g * 64;
              if (sl < ni) {
                const long long sz = rp->inner_size[sl];
                long long dig;
                rem = apx_divmod(rem, sz, &dig);
                src[sl] += (rp->inner_row[sl] + dig) * 256;
              }
            }
          }
          if (row_ok) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
              for (int sl = 0; sl < APEX_MAX_SLOTS; ++sl) {
                if (sl >= ni) break;
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src[sl] + c * 8));
                const float2 f0 = unpack2<PF>(v.x), f1 = unpack2<PF>(v.y), f2 = unpack2<PF>(v.z), f3 = unpack2<PF>(v.w);
                acc[0] += f0.x; acc[1] += f0.y; acc[2] += f1.x; acc[3] += f1.y;
                acc[4] += f2.x; acc[5] += f2.y; acc[6] += f3.x; acc[7] += f3.y;
              }
              R[c * 4 + 0] = pack2<PF>(acc[0], acc[1]);
              R[c * 4 + 1] = pack2<PF>(acc[2], acc[3]);
              R[c * 4 + 2] = pack2<PF>(acc[4], acc[5]);
              R[c * 4 + 3] = pack2<PF>(acc[6], acc[7]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) R[c] = 0u;
          }
          need_r = false;
        }
        // ---- layer 1 of tile s: stage g of a_1
        const int rs = (int)(s & (TC_OROW_SLOTS - 1));
        ok = ok && mbar_wait(bar(B_OFULL(rs)), (uint32_t)((s / TC_OROW_SLOTS) & 1), abort_flag, err);
        const unsigned char *prow = sm + LY::OROW + (uint32_t)rs * 512u + (uint32_t)g * 128u;
        // 16-bit: stage g (K quarter g) of the single a_1 buffer. FP8: K half g / 2 of buffer s & 1
        // (two tiles in flight), this quarter's 64 bytes at byte 64 (g & 1) of the 128-byte rows.
        const int stg = F8 ? (int)((s & 1u) * 2u + (unsigned)(g >> 1)) : g;
        const uint32_t use = F8 ? (s >> 1) : s;  // how many times this stage was filled before
        ok = ok && mbar_wait(bar(B_EMPTY(stg)), (use & 1u) ^ 1u, abort_flag, err);
        if (ok) {
          unsigned char *stage = sm + LY::A1 + (uint32_t)stg * LY::STAGE + row_off;
          if (!F8) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              uint4 pv = make_uint4(0u, 0u, 0u, 0u);
              if (!IDS) pv = *reinterpret_cast<const uint4 *>(prow + c * 16);  // 1-slot reactions: the zero row
              const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w};
              uint32_t out[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) out[e] = act2<ACT, PF>(add2<PF>(R[c * 4 + e], pw[e]));
              *reinterpret_cast<uint4 *>(stage + (uint32_t)((c ^ (m & 7)) * 16)) = make_uint4(out[0], out[1], out[2], out[3]);
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {  // 16 K elements (16 bytes) per piece
              uint32_t q[4];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int c = 2 * cc + h;
                uint4 pv = make_uint4(0u, 0u, 0u, 0u);
                if (!IDS) pv = *reinterpret_cast<const uint4 *>(prow + c * 16);
                const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w};
                uint32_t out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) out[e] = fma2<PF>(act2<ACT, PF>(add2<PF>(R[c * 4 + e], pw[e])), a1s, 0u);
                q[2 * h] = e4m3x4(out[0], out[1]);
                q[2 * h + 1] = e4m3x4(out[2], out[3]);
              }
              const int piece = (g & 1) * 4 + cc;
              *reinterpret_cast<uint4 *>(stage + (uint32_t)((piece ^ (m & 7)) * 16)) = make_uint4(q[0], q[1], q[2], q[3]);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(bar(B_FULL(stg)));
            mbar_arrive(bar(B_OEMPTY(rs)));
          }
        }
        ++tile;
        if (--left == 0) {
          more = tile < rend;
          while (!more && L.pool_ctr && pool_next(n_ring, tile, rend, true)) more = tile < rend;
          need_r = more;
        }
      }
      // ---- layer-2 activation of tile s - 1 (columns [64g, 64g + 64) of its accumulator)
      if (ok && s >= 1) {
        const unsigned jj = s - 1;
        const int buf = (int)(jj & 1);
        ok = mbar_wait(bar(B_D2FULL(buf)), (uint32_t)((jj >> 1) & 1), abort_flag, err);
        if (ok) {
          tc_fence_after();
          const uint32_t col = lane_base + (uint32_t)buf * 256u + (uint32_t)g * 64u;
          const uint32_t *bh = reinterpret_cast<const uint32_t *>(b2s) + g * 32;
          // 16 accumulator columns at a time -> 8 packed 16-bit pairs written over columns already
          // read (a_2 of this quarter lands in its first 32 columns); one load of lookahead
          uint32_t va[16], vb[16];
          tmem_ld16(col, va);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t(&v)[16] = (c & 1) ? vb : va;
            uint32_t(&vn)[16] = (c & 1) ? va : vb;
            tmem_wait_ld_dep16(v);
            if (c + 1 < 4) tmem_ld16(col + (uint32_t)(c + 1) * 16u, vn);
            uint32_t pk[8];
            if (!F8) {
#pragma unroll
              for (int e4 = 0; e4 < 2; ++e4) {
                const uint4 bb = *reinterpret_cast<const uint4 *>(bh + c * 8 + 4 * e4);
                const uint32_t bw[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                {
                  const uint32_t hh = add2<PF>(
                      pack2<PF>(__uint_as_float(v[8 * e4 + 2 * e]), __uint_as_float(v[8 * e4 + 2 * e + 1])), bw[e]);
                  pk[4 * e4 + e] = (ACT == APEX_ACT_SILU && PF == 0 && ((TC_EX2_PAIRS >> (4 * e4 + e)) & 1u))
                                       ? silu2_ex2_bf16(hh)
                                       : act2<ACT, PF>(hh);
                }
              }
              tmem_st8(col + (uint32_t)c * 8u, pk);
            } else {
              // FP8 layer 2: dequantize per output channel (h = D s_2[n] + b_2[n]) in FP32, then the
              // FP16 activation; a_2 stays FP16 for layer 3
              const int n0 = g * 64 + c * 16;
#pragma unroll
              for (int e4 = 0; e4 < 4; ++e4) {
                const float4 sc = *reinterpret_cast<const float4 *>(s2s + n0 + 4 * e4);
                const float4 bb = *reinterpret_cast<const float4 *>(b2s + n0 + 4 * e4);
                pk[2 * e4] = act2<ACT, PF>(pack2<PF>(fmaf(__uint_as_float(v[4 * e4]), sc.x, bb.x),
                                                     fmaf(__uint_as_float(v[4 * e4 + 1]), sc.y, bb.y)));
                pk[2 * e4 + 1] = act2<ACT, PF>(pack2<PF>(fmaf(__uint_as_float(v[4 * e4 + 2]), sc.z, bb.z),
                                                         fmaf(__uint_as_float(v[4 * e4 + 3]), sc.w, bb.w)));
              }
              tmem_st8(col + (uint32_t)c * 8u, pk);
            }
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_A2FULL(buf)));
        }
      }
      if (!produce) break;
    }
  } else if (warp == TC_LOAD_WARP) {
    // ------------------------------------------------------------ outer-row loader (bulk TMA)
    if (lane == 0 && IDS) {  // id lists have no outer rows: keep the ring's phases
      for (long long j = 0; j < t_end - t_begin; ++j) {
        const int rs = (int)(j & (TC_OROW_SLOTS - 1));
        if (!mbar_wait(bar(B_OEMPTY(rs)), (uint32_t)(((j / TC_OROW_SLOTS) & 1) ^ 1), abort_flag, err)) break;
        mbar_arrive(bar(B_OFULL(rs)));
      }
    } else if (lane == 0) {
      long long j = 0;
      bool ok = true;
      long long ra = t_begin, rb = t_end;  // current range: this CTA's own, then tail-pool chunks
      unsigned n_ring = 0;
      for (;;) {
      for (long long tile = ra; ok && tile < rb;) {
        const TileRun I = apx_tile_run(L, T.rx, tile, rb);
        tile += I.o_end - I.o_begin;
        const long long orow = I.rp->outer_row;
        for (long long o = I.o_begin; o < I.o_end; ++o, ++j) {
          const int rs = (int)(j & (TC_OROW_SLOTS - 1));
          if (!mbar_wait(bar(B_OEMPTY(rs)), (uint32_t)(((j / TC_OROW_SLOTS) & 1) ^ 1), abort_flag, err)) {
            ok = false;
            break;
          }
          // the outer synthon's row; a reaction without an outer slot (one slot) gets the table's
          // zero row (row n_rows), so that the math warps add a row whatever the reaction
          const unsigned short *src = T.P16[PF] + (orow >= 0 ? orow + o : T.n_rows) * 256;
          mbar_expect_tx(bar(B_OFULL(rs)), 512u);
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 512, [%2];" ::"r"(
                  sbase + LY::OROW + (uint32_t)rs * 512u),
              "l"(src), "r"(bar(B_OFULL(rs)))
              : "memory");
        }
      }
      if (!ok || !L.pool_ctr) break;
      // claim the next chunk of the tail pool (or learn that it is empty) and publish it to the
      // other roles; the claim runs a few tiles ahead of the math warps (the outer-row ring's depth)
      const long long a = L.pool_first + (long long)atomicAdd(L.pool_ctr, (unsigned long long)L.pool_chunk);
      ra = a < L.total_tiles ? a : -1;
      rb = a < L.total_tiles ? (a + L.pool_chunk < L.total_tiles ? a + L.pool_chunk : L.total_tiles) : -1;
      if (!pool_publish(n_ring, ra, rb) || ra < 0) break;
      }
    }
    __syncwarp();
  } else if (warp == TC_MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      if (mbar_wait(bar(B_W), 0, abort_flag, err)) {
        tc_fence_after();
        const uint32_t a1 = sbase + LY::A1, w2 = sbase + LY::W2;
        bool ok = true;
        {
          long long n_tiles = t_end - t_begin, pa = 0, pb = 0;  // own range, then tail-pool ranges
          unsigned n_ring = 0;
          bool have = true;
          for (long long j = 0;; ++j) {  // this CTA's tiles, in order
            while (j == n_tiles && (have = (L.pool_ctr && pool_next(n_ring, pa, pb, false)))) n_tiles += pb - pa;
            if (!have) break;
            const int buf = (int)(j & 1);
            if (!mbar_wait(bar(B_D2EMPTY(buf)), (uint32_t)(((j >> 1) & 1) ^ 1), abort_flag, err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d2 = tmem + (uint32_t)buf * 256u;
            if (!F8) {  // four K-quarter stages, four K16 MMAs each
              constexpr uint32_t ID2 = idesc_16(128, 256, FMT);
              for (int kc = 0; kc < 4; ++kc) {
                if (!mbar_wait(bar(B_FULL(kc)), (uint32_t)(j & 1), abort_flag, err)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                  mma_ss(d2, sw128_desc(a1 + (uint32_t)kc * LY::STAGE + (uint32_t)ks * 32u),
                         sw128_desc(w2 + (uint32_t)kc * 32768u + (uint32_t)ks * 32u), ID2, (kc | ks) != 0);
                mma_commit(bar(B_EMPTY(kc)));
              }
            } else {  // two K-half stages of buffer j & 1, four K32 MMAs each
              constexpr uint32_t ID2 = idesc_e4m3(128, 256);
              for (int kc = 0; kc < 2; ++kc) {
                const int stg = (int)(j & 1) * 2 + kc;
                if (!mbar_wait(bar(B_FULL(stg)), (uint32_t)((j >> 1) & 1), abort_flag, err)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                  mma_ss_f8(d2, sw128_desc(a1 + (uint32_t)stg * LY::STAGE + (uint32_t)ks * 32u),
                            sw128_desc(w2 + (uint32_t)kc * 32768u + (uint32_t)ks * 32u), ID2, (kc | ks) != 0);
                mma_commit(bar(B_EMPTY(stg)));
              }
            }
            if (!ok) break;
            mma_commit(bar(B_D2FULL(buf)));
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == TC_L3_WARP) {
    // ------------------------------------------------------------ layer-3 issuer
    // Issues each tile's layer-3 MMAs as soon as its a_2 is complete, so that they neither queue
    // behind the MMA warp's layer-2 work of the next tile nor wait for the query epilogue.
    if (lane == 0 && mbar_wait(bar(B_W), 0, abort_flag, err)) {
      const uint32_t w3 = sbase + LY::W3;
      long long n_tiles = t_end - t_begin, pa = 0, pb = 0;  // own range, then tail-pool ranges
      unsigned n_ring = 0;
      bool have = true;
      for (long long j = 0;; ++j) {
        while (j == n_tiles && (have = (L.pool_ctr && pool_next(n_ring, pa, pb, false)))) n_tiles += pb - pa;
        if (!have) break;
        const int buf = (int)(j & 1);
        if (!mbar_wait(bar(B_A2FULL(buf)), (uint32_t)((j >> 1) & 1), abort_flag, err)) break;
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)buf * 256u;
        constexpr uint32_t ID3 = idesc_16(128, 16, PF);
#pragma unroll
        for (int ks = 0; ks < 16; ++ks)  // K block ks (16 wide) of a_2: quarter ks / 4, 8 columns each
          mma_ts(dcol + tc_d3_col(ks % TC_L3_CHAINS), dcol + (uint32_t)(ks >> 2) * 64u + (uint32_t)(ks & 3) * 8u,
                 sw128_desc(w3 + (uint32_t)(ks >> 2) * 2048u + (uint32_t)(ks & 3) * 32u), ID3, ks >= TC_L3_CHAINS);
        mma_commit(bar(B_D3FULL(buf)));
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ query warps (0-3)
    // read the head outputs of each tile (D3), release its accumulator buffer, apply the queries
    const int r = tid;  // tile row == TMEM lane
    // every query of a library has the library's objective count
    const int qp_n_obj = L.qmask_all ? qp[__ffsll((long long)L.qmask_all) - 1].n_obj : APEX_MAX_OBJECTIVES;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    if constexpr (IDS) {  // outputs of the listed compounds, FP32, row-major [n x n_out]
      for (long long j = 0; j < t_end - t_begin; ++j) {
        const int buf = (int)(j & 1);
        if (!mbar_wait(bar(B_D3FULL(buf)), (uint32_t)((j >> 1) & 1), abort_flag, err)) break;
        tc_fence_after();
        float out[16];
#pragma unroll
        for (int n = 0; n < 16; ++n) out[n] = b3s[n];
#pragma unroll
        for (int c = 0; c < TC_L3_CHAINS; ++c) {
          uint32_t pa[16];
          tmem_ld16(lane_base + (uint32_t)buf * 256u + tc_d3_col(c), pa);
          tmem_wait_ld_dep16(pa);
#pragma unroll
          for (int n = 0; n < 16; ++n) out[n] += __uint_as_float(pa[n]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_D2EMPTY(buf)));
        const long long i = (t_begin + j) * APX_TILE + r;
        if (i < n_ids) {
          if (L.dump_base >= 0) {  // start-threshold sample of query slot dump_base: its key
            const QuerySlot *Q = slots + L.dump_base;
            const int n_obj = Q->n_obj;
            float f = 0.f;
#pragma unroll
            for (int o = 0; o < 16; ++o)
              if (o < n_obj) f = fmaf(Q->w[o], out[o], f);
            bool feasible = true;
            for (int c = 0; c < Q->n_cons; ++c) {
              const float v = apx_sel(out, Q->cons_idx[c]);
              feasible = feasible && v >= Q->lo_x[c] && v <= Q->hi_x[c];
            }
            reinterpret_cast<unsigned *>(L.dump)[i] = feasible ? apx_key_bits(f) : 0u;
          } else {
#pragma unroll
            for (int n = 0; n < 16; ++n)
              if (n < T.n_out) L.dump[i * T.n_out + n] = out[n];
          }
        }
      }
    }
    long long j = 0;
    bool ok = !IDS;
    long long ra = t_begin, rb = t_end;  // own range, then tail-pool ranges
    unsigned n_ring = 0;
    for (long long tile = ra; ok;) {
      if (tile >= rb) {  // range done: the next tail-pool range, if any
        if (!L.pool_ctr || !pool_next(n_ring, ra, rb, true)) break;
        tile = ra;
        continue;
      }
      const TileRun I = apx_tile_run(L, T.rx, tile, rb);
      const long long run_tile0 = tile - I.o_begin;  // launch tile of outer index o: run_tile0 + o
      // this run's query slots, as a list
      unsigned char *qlist = sm + LY::QLIST + (uint32_t)warp * APEX_MAX_ACTIVE;
      int nq = 0;
      if (lane == 0) {
        for (unsigned long long m = I.qmask; m; m &= m - 1) qlist[nq++] = (unsigned char)(__ffsll((long long)m) - 1);
      }
      nq = __shfl_sync(0xffffffffu, nq, 0);
      __syncwarp();
      tile += I.o_end - I.o_begin;
      const RxnPlan *rp = I.rp;
      const long long q = I.q0 + r;
      const bool valid = q < rp->n_inner;
      const long long id_row = rp->id_first + q * rp->inner_stride;  // id = id_row + o * outer_stride
      const long long ostride = rp->outer_stride;
      for (long long o = I.o_begin; o < I.o_end; ++o, ++j) {
        const int buf = (int)(j & 1);
        if (!mbar_wait(bar(B_D3FULL(buf)), (uint32_t)((j >> 1) & 1), abort_flag, err)) { ok = false; break; }
        tc_fence_after();
        // the four layer-3 partial sums, one chain (16 columns) per load
        float out[16];
#pragma unroll
        for (int n = 0; n < 16; ++n) out[n] = b3s[n];
#pragma unroll
        for (int c = 0; c < TC_L3_CHAINS; ++c) {
          uint32_t pa[16];
          tmem_ld16(lane_base + (uint32_t)buf * 256u + tc_d3_col(c), pa);
          tmem_wait_ld_dep16(pa);
#pragma unroll
          for (int n = 0; n < 16; ++n) out[n] += __uint_as_float(pa[n]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_D2EMPTY(buf)));
        const long long id = id_row + o * ostride;
        if (L.mode == 0) {
          tc_apply_queries<FEWQ>(qp, slots, qlist, nq, valid, id, out, qp_n_obj);
        } else if (L.mode == 1) {
          if (valid && id >= L.dump_base && id < L.dump_base + L.dump_n) {
#pragma unroll
            for (int n = 0; n < 16; ++n)
              if (n < T.n_out) L.dump[(id - L.dump_base) * T.n_out + n] = out[n];
          }
        } else {
          const long long slot = (run_tile0 + o) * APX_TILE + r;
          if (slot < L.dump_n) {
            L.dump_ids[slot] = valid ? id : -1;
#pragma unroll
            for (int n = 0; n < 16; ++n)
              if (n < T.n_out) L.dump[slot * T.n_out + n] = out[n];
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == TC_L3_WARP && lane == 0 && *abort_flag) {
    // after an abort, layer-3 MMAs of this issuer may still be in flight: wait (bounded)
    tc_fence_after();
    mma_commit(bar(B_DRAIN3));
    const unsigned long long t0 = globaltimer();
    while (!mbar_try(bar(B_DRAIN3), 0) && globaltimer() - t0 < 2000000000ull) {
    }
  }
  if (warp == TC_MMA_WARP) {
    tc_fence_after();
    if (*abort_flag && lane == 0) {
      // after an abort, MMAs may still be in flight: wait (bounded) until they retire
      mma_commit(bar(B_DRAIN));
      const unsigned long long t0 = globaltimer();
      while (!mbar_try(bar(B_DRAIN), 0) && globaltimer() - t0 < 2000000000ull) {
      }
    }
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

size_t apx_tc_smem_bytes() { return TcL<1>::SMEM; }

template <int ACT, int FMT, bool FEWQ, bool IDS = false>
static cudaError_t tc_launch_q(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                               cudaStream_t st) {
  static bool attr = false;  // per instantiation
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_tc_head<ACT, FMT, FEWQ, IDS>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, TcL<FMT>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (grid <= 0) return cudaSuccess;
  apx_count_launch();
  k_tc_head<ACT, FMT, FEWQ, IDS><<<grid, TC_THREADS, TcL<FMT>::SMEM, st>>>(L, T, slots, err);
  return cudaGetLastError();
}
template <int ACT, int FMT>
static cudaError_t tc_launch_one(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                                 cudaStream_t st) {
  if (__builtin_popcountll(L.qmask_all) <= TC_FEWQ) return tc_launch_q<ACT, FMT, true>(L, T, slots, err, grid, st);
  return tc_launch_q<ACT, FMT, false>(L, T, slots, err, grid, st);
}

template <int FMT>
static cudaError_t tc_launch_fmt(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                                 cudaStream_t st) {
  if (T.act == APEX_ACT_SILU) return tc_launch_one<APEX_ACT_SILU, FMT>(L, T, slots, err, grid, st);
  if (T.act == APEX_ACT_RELU) return tc_launch_one<APEX_ACT_RELU, FMT>(L, T, slots, err, grid, st);
  return tc_launch_one<APEX_ACT_IDENTITY, FMT>(L, T, slots, err, grid, st);
}

// fmt: 0 = BF16 tables and arithmetic, 1 = FP16, 2 = FP8 e4m3 operands (FP16 table and activations)
cudaError_t apx_launch_tc(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                          cudaStream_t st, int fmt) {
  if (fmt == 0) return tc_launch_fmt<0>(L, T, slots, err, grid, st);
  if (fmt == 1) return tc_launch_fmt<1>(L, T, slots, err, grid, st);
  return tc_launch_fmt<2>(L, T, slots, err, grid, st);
}

template <int FMT>
static cudaError_t tc_launch_ids_fmt(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                                     cudaStream_t st) {
  if (T.act == APEX_ACT_SILU) return tc_launch_q<APEX_ACT_SILU, FMT, true, true>(L, T, slots, err, grid, st);
  if (T.act == APEX_ACT_RELU) return tc_launch_q<APEX_ACT_RELU, FMT, true, true>(L, T, slots, err, grid, st);
  return tc_launch_q<APEX_ACT_IDENTITY, FMT, true, true>(L, T, slots, err, grid, st);
}

// Outputs of n listed compounds (ids: device, bit 62 ignored) in the reduced-precision pass format
// fmt, as FP32 rows out[n x n_out] (device). One tile of 128 ids per CTA step. With spec_slot >= 0
// the kernel applies that query slot's exact boxes and objective instead and writes one key per
// compound into out (as unsigned: order-preserving objective bits, 0 = infeasible).
cudaError_t apx_launch_tc_ids(const DevTables &T, const long long *ids, long long n, float *out, int *err, int n_sm,
                              cudaStream_t st, int fmt, QuerySlot *slots, int spec_slot, const unsigned *n_dev) {
  if (n <= 0) return cudaSuccess;
  LaunchPlan L;
  memset(&L, 0, sizeof(L));
  L.mode = 3;
  L.total_tiles = (n + APX_TILE - 1) / APX_TILE;
  L.dump = out;
  L.dump_ids = const_cast<long long *>(ids);
  L.dump_n = n;
  L.dump_n_dev = n_dev;
  L.dump_base = spec_slot >= 0 && slots ? spec_slot : -1;
  const int grid = (int)std::min<long long>(L.total_tiles, n_sm);
  if (fmt == 0) return tc_launch_ids_fmt<0>(L, T, slots, err, grid, st);
  if (fmt == 1) return tc_launch_ids_fmt<1>(L, T, slots, err, grid, st);
  return tc_launch_ids_fmt<2>(L, T, slots, err, grid, st);
}

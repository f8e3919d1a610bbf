// mlp_lay.cu -- (a1, reverse mode, layered) residual network value f_D and
// input Jacobian J_D of every node, one layer of every node at a time.
//
// The fused kernels (mlp_rev.cu, mlp_rev2.cu) carry a tile of nodes through
// all layers inside one CTA (pair), so each GEMM waits for the previous
// layer's epilogue.  Here every layer is one GEMM over all nodes, its
// activations passing through HBM/L2:
//   input      a_1 = tanh(W_0 z + b_0)                           (tcgen05, K = 17 -> 32)
//   forward    a_{l+1} = tanh(W_l a_l + b_l)                     (tcgen05)
//   output     f_D = W_L a_L + b_L                               (SIMT)
//   adjoints   D_L = d_L (.) W_L' (three columns per node)       (SIMT)
//   backward   D_l = d_l (.) (W_l' D_{l+1}), d_l = 1 - a_l^2     (tcgen05)
//   Jacobian   J_D = W_0' D_1                                    (tcgen05)
// with the split-BF16 arithmetic of the fused kernels: BF16 weights (W_0'
// split hi + lo), activations and adjoints stored as BF16 hi + lo pairs (two
// MMAs per K step, FP32 accumulation).  Every layer's activations are kept
// and d_l is recomputed from them in the backward epilogues (a stored d_l
// would be one more write of every layer).  Layout: node-major rows,
// X [node][hs] for values, [node * 3 + r][hs] for adjoints, so both operands
// are K-major TMA tiles (128 B swizzle) and an epilogue lane (one neuron)
// stores consecutive neurons of a node across the warp.
// Tiles: M = 128 rows x N = 256 nodes (forward) or 80 nodes x 3 adjoints
// (backward, Jacobian); persistent CTAs, K in stages of 64, two TMEM
// accumulators so that the epilogue of one tile overlaps the next's MMAs.
#include <cuda_fp8.h>

#include <algorithm>

#include "tc_common.cuh"
#include "tc_pair.cuh"

namespace rtn {
namespace {

// K per stage: one 64 B row of BF16 (64 B swizzle), so that four stages of
// every mode fit and the TMA runs four K blocks ahead of the MMAs (with two
// stages of 128 B rows the GEMMs waited on each stage's DRAM latency)
constexpr int LY_KB = 32;
constexpr uint32_t LY_SBO = 512;   // 8 rows x 64 B between 8-row groups
constexpr uint32_t LY_SWZ = 4;     // descriptor swizzle mode: 64 B
constexpr uint32_t LY_A_BYTES = 128u * LY_KB * 2u;  // one 128-row weight tile
constexpr int LY_NF = 256;                          // forward tile: nodes
constexpr int LY_NBN = 80;                          // backward tile: nodes
constexpr int LY_NODE_PAD = 1280;                   // node rows padded to a multiple of both
constexpr int LY_THREADS = 320;                     // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int LY_EPI_WARPS = 8;                     // two per TMEM lane quarter, alternate column chunks
constexpr int LY_STAGES = 4;
constexpr uint32_t LY_TMEM_COLS = 512;
// FWD forward layer; BWD backward layer; JD the W_0' Jacobian; BW0 the
// first backward layer with the last-layer adjoints folded into its weights
// (M_r = W_{L-2}' diag(W_L[r]), B = d_{L-1}), see mlp_lay_launch
// IN the input layer as a GEMM (W_0 hi / lo against z hi / lo, K = 17
// padded to 32) with the forward epilogue
enum { LY_FWD = 0, LY_BWD = 1, LY_JD = 2, LY_BW0 = 3, LY_IN = 4 };

// F8: the FP8 variant of the forward and backward hidden GEMMs (RTN_FP8):
// e4m3 weights against activations / adjoints held as three e4m3 pieces, K
// blocks of 64 one-byte elements (the same 64 B rows), three B tiles per
// stage and three kind::f8f6f4 MMAs per K step
template <int MODE, bool F8 = false>
struct Ly {
  static constexpr bool ACT = MODE == LY_FWD || MODE == LY_IN;      // tanh epilogue
  static constexpr bool BYNODE = ACT || MODE == LY_BW0;             // one column per node
  static constexpr int N = BYNODE ? LY_NF : 3 * LY_NBN;            // MMA N
  static constexpr int NODES = BYNODE ? LY_NF : LY_NBN;            // nodes per tile
  static constexpr int NA = (MODE == LY_JD || MODE == LY_BW0 || MODE == LY_IN) ? 2 : 1;  // weight tiles (hi, lo)
  static constexpr int NB = F8 ? 3 : 2;                             // B tiles: pieces
  static constexpr int KB = F8 ? 64 : LY_KB;                        // K elements per stage
  // split-BF16 backward: the tile's activations a_l (hi, lo) reach the
  // epilogue through shared memory, one 16-node group per buffer of a ring of
  // three loaded by TMA from an eleventh warp (global loads of 2 B per lane
  // were the epilogue's largest cost)
  // The first backward GEMM (its d_{L-2} from a_{L-2}) reads them the same
  // way, 16-node chunks through a ring of ten.
  static constexpr bool STAGE_ACT = (MODE == LY_BWD || MODE == LY_BW0) && !F8;
  // split-BF16 backward and forward: the outputs (adjoints D_l, activations
  // a_{l+1}) leave through shared memory, each group of four epilogue warps
  // (one per TMEM lane quarter) staging its rows x 128 neurons (hi, lo; two
  // buffers per group) for TMA tensor stores (2-byte stores per lane
  // competed with the operand loads: backward GEMM 0.51 vs 0.40 ms per
  // launch without them).  Backward: 24 rows (8 nodes x 3 adjoints) per
  // half-group; forward: a 16-node chunk.
  static constexpr bool STAGE_OUT = (MODE == LY_BWD || MODE == LY_FWD) && !F8;
  // the first backward GEMM trades a stage for a deeper activation ring
  // (its epilogue, two activation loads per output, bounds it; three stages
  // and ten ring buffers 0.586 -> 0.567 ms per launch)
  static constexpr int STAGES = MODE == LY_BW0 ? 3 : LY_STAGES;
  // epilogue warps: 4 per TMEM lane quarter in the forward and input GEMMs
  // (their epilogue, tanh and stores with no loads, bounds them: split-BF16
  // forward GEMM 0.184 -> 0.174 ms, input 0.157 -> 0.111, FP8 forward 0.195
  // -> 0.165 with 16 instead of 8), else 2
  static constexpr int EPI = (MODE == LY_FWD || MODE == LY_IN) ? 16 : LY_EPI_WARPS;
  static constexpr int THREADS = 64 + 32 * EPI + (STAGE_ACT ? 32 : 0);
  static constexpr int ACT_RING = MODE == LY_BW0 ? 10 : 3;            // ring buffers
  static constexpr int ACT_CHUNKS = NODES / 16;                      // 16-node chunks per tile
  static constexpr int ACT_READERS = MODE == LY_BW0 ? LY_EPI_WARPS / 2 : LY_EPI_WARPS;  // warps reading a chunk
  static constexpr int OUT_GROUPS = EPI / 4;                                         // staging groups
  static constexpr uint32_t OUT_BUF = MODE == LY_BWD ? 2u * 24u * 128u * 2u : 2u * 16u * 128u * 2u;  // bytes
  static constexpr uint32_t OUT_BYTES = STAGE_OUT ? 2u * OUT_GROUPS * OUT_BUF : 0u;
  static constexpr int OUT_BARS = STAGE_OUT ? 4 * OUT_GROUPS : 0;
};
// one ring buffer: the activations of 16 nodes x 128 neurons, hi then lo
constexpr uint32_t LY_ACT_BYTES = 2u * 16u * 128u * 2u;
// one output staging buffer: 24 adjoint rows x 128 neurons, hi then lo
constexpr uint32_t LY_OUT_BYTES = 2u * 24u * 128u * 2u;
template <int MODE, bool F8 = false>
__host__ __device__ constexpr uint32_t ly_b_bytes() { return (uint32_t)Ly<MODE>::N * 64u; }
template <int MODE, bool F8 = false>
__host__ __device__ constexpr uint32_t ly_stage() {
  return Ly<MODE, F8>::NA * LY_A_BYTES + Ly<MODE, F8>::NB * ly_b_bytes<MODE>();
}
template <int MODE, bool F8 = false>
__host__ __device__ constexpr size_t ly_smem() {
  return Ly<MODE, F8>::STAGES * ly_stage<MODE, F8>() +
         (Ly<MODE, F8>::STAGE_ACT ? Ly<MODE, F8>::ACT_RING * LY_ACT_BYTES : 0) +
         Ly<MODE, F8>::OUT_BYTES + 1024 + 512;
}
static_assert(ly_b_bytes<LY_FWD>() % 1024 == 0 && ly_b_bytes<LY_BWD>() % 1024 == 0, "1 KB aligned tiles");
static_assert(ly_smem<LY_JD>() <= 232448 && ly_smem<LY_FWD>() <= 232448 && ly_smem<LY_BW0>() <= 232448 &&
                  ly_smem<LY_FWD, true>() <= 232448 && ly_smem<LY_BWD, true>() <= 232448 &&
                  ly_smem<LY_BWD>() <= 232448,
              "shared memory");
static_assert(Ly<LY_BWD>::OUT_BUF == LY_OUT_BYTES, "backward staging buffer");
static_assert(ly_stage<LY_BWD>() % 1024 == 0 && ly_stage<LY_BW0>() % 1024 == 0 && LY_ACT_BYTES % 1024 == 0 &&
                  LY_OUT_BYTES % 1024 == 0,
              "1 KB aligned activation and output buffers");

struct LyMaps {
  CUtensorMap bh, bl, b3;  // activations / adjoints hi, lo (F8: hi, mid, lo)
  CUtensorMap sh, sl;      // split-BF16 backward: the activations a_l hi, lo, box 128 x 16
  CUtensorMap oh, ol;      // split-BF16 output stores: backward D_l hi, lo (box 128 x 24), forward a_{l+1} (128 x 16)
};

struct LyArgs {
  int a_row0;     // weight row of M tile 0 in the stacked weights
  int b_row0;     // FWD: first row of the source layer in the stacked activations
  int a_lo;       // JD: row offset of the lo weights
  int m_rows;     // real output rows
  int mts;        // M tiles
  int mtpr;       // BW0: M tiles per output component r
  int nkb;        // K blocks
  int n_nodes, n_groups, hs;
  const float* bias;   // FWD: bias of the produced layer
  __nv_bfloat16* dh;   // FWD, last hidden layer: its d as BF16 hi + lo (the
  __nv_bfloat16* dl;   //      B operand of the folded first backward GEMM)
  int act_row0;        // split-BF16 BWD / BW0: row of node 0 of a_l in the stacked activations
  int out_row0;        // split-BF16 FWD: row of node 0 of the produced layer in the stacked activations
  const __nv_bfloat16* ah;  // BW0 / BWD: a_l of the adjoint's layer [node][hs]
  const __nv_bfloat16* al;  //            hi / lo, d_l = 1 - a_l^2
  __nv_bfloat16* yh;   // FWD / BWD outputs
  __nv_bfloat16* yl;
  float* JD;           // JD output [node][3][17]
  int* err;
  long long wait_cycles;  // budget of every bounded pipeline wait [SM cycles]
  int stall;              // fault injection: the TMA producer first waits on a barrier nothing completes
  // RTN_FP8: F8 GEMMs scale the accumulator by sc (weight scale over the
  // B operand's scale); y8 (if set) receives the output as three e4m3
  // pieces of (value * s8); a8: the F8 backward GEMM's a_l pieces (a * 448)
  float sc, s8;
  uint8_t *y8h, *y8m, *y8l;
  const uint8_t *a8h, *a8m, *a8l;
};

// four values as e4m3 pieces, four codes per word (byte k = value k): wh the
// roundings, wm the roundings of the residuals, wl of the residuals' residuals
__device__ __forceinline__ void split3x4(const float* v, uint32_t& wh, uint32_t& wm, uint32_t& wl) {
  float r[4] = {v[0], v[1], v[2], v[3]};
  uint32_t w[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const uint32_t a = __nv_cvt_float2_to_fp8x2(make_float2(r[0], r[1]), __NV_SATFINITE, __NV_E4M3);
    const uint32_t b = __nv_cvt_float2_to_fp8x2(make_float2(r[2], r[3]), __NV_SATFINITE, __NV_E4M3);
    w[p] = a | (b << 16);
    if (p < 2) {
      const float2 fa = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)a, __NV_E4M3)));
      const float2 fb = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)b, __NV_E4M3)));
      r[0] -= fa.x; r[1] -= fa.y; r[2] -= fb.x; r[3] -= fb.y;
    }
  }
  wh = w[0]; wm = w[1]; wl = w[2];
}

// the four values of a word of e4m3 codes
__device__ __forceinline__ void e4m3x4(uint32_t w, float* f) {
  const float2 a = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3)));
  const float2 b = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3)));
  f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
}

// 4 x 4 byte transpose across the lanes of a quad (t = lane & 3): lane t
// holds a word whose byte k is element (t, k); returns the word whose byte
// k is element (k, t).  An epilogue lane owns one output row for several
// nodes; after the transpose it owns four rows of one node, which it stores
// (or, for loads, the reverse) as one 4-byte word.
__device__ __forceinline__ uint32_t quad_transpose(uint32_t x, int t) {
  const uint32_t y = __shfl_xor_sync(0xffffffffu, x, 2);
  x = (t & 2) ? __byte_perm(x, y, 0x3276) : __byte_perm(x, y, 0x5410);
  const uint32_t z = __shfl_xor_sync(0xffffffffu, x, 1);
  return (t & 1) ? __byte_perm(x, z, 0x3715) : __byte_perm(x, z, 0x6240);
}

// 4 m .. 4 m + 3 of a lane's values (one row, consecutive nodes) as e4m3
// pieces, stored through quad transposes: lane t writes the word of rows
// i & ~3 .. + 3 of node n0 + t at dst_p + (n0 + t) * stride + (i & ~3)
__device__ __forceinline__ void store_pieces4(const float* v, int t, int n0, int n_nodes, size_t stride, int i4,
                                              uint8_t* dh, uint8_t* dm, uint8_t* dl) {
  uint32_t wh, wm, wl;
  split3x4(v, wh, wm, wl);
  wh = quad_transpose(wh, t);
  wm = quad_transpose(wm, t);
  wl = quad_transpose(wl, t);
  if (n0 + t < n_nodes) {
    const size_t o = (size_t)(n0 + t) * stride + i4;
    *reinterpret_cast<uint32_t*>(dh + o) = wh;
    *reinterpret_cast<uint32_t*>(dm + o) = wm;
    *reinterpret_cast<uint32_t*>(dl + o) = wl;
  }
}

__device__ __forceinline__ void split_bf(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// the activation pairs a_l of the 8 nodes that the warp of half H stores in
// a 16-node group of a backward tile, from the group's shared-memory buffer
// [16 nodes][128 neurons] (hi, then lo at +16 x 128), column col
template <int H>
__device__ __forceinline__ void bwd_load_s(const __nv_bfloat16* __restrict__ sh, int col, __nv_bfloat16 (&ph)[8],
                                           __nv_bfloat16 (&pl)[8]) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const int o = (8 * H + kk) * 128 + col;
    ph[kk] = sh[o];
    pl[kk] = sh[16 * 128 + o];
  }
}

// backward epilogue of one 16-node group (48 accumulator columns, node k
// in columns 3k .. 3k + 2): the warp of half H computes nodes 8H .. 8H + 7,
// D = acc * d with d = 1 - a^2 computed once per node from the loaded pairs,
// into the half's staging buffer [24 rows (node, r)][128 neurons] hi, then
// lo, column col.  Rows of nodes past the end and columns past the layer's
// width are written as zeros (the values the buffer's padding holds).
template <int H>
__device__ __forceinline__ void bwd_group_s(const float (&v)[48], const __nv_bfloat16 (&ph)[8],
                                            const __nv_bfloat16 (&pl)[8], int node_g, int n_nodes, bool active,
                                            __nv_bfloat16* __restrict__ so, int col) {
  float dv[8];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const float av = __bfloat162float(ph[kk]) + __bfloat162float(pl[kk]);
    dv[kk] = (active && node_g + 8 * H + kk < n_nodes) ? 1.0f - av * av : 0.0f;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      __nv_bfloat16 h, l;
      split_bf(v[3 * (8 * H + kk) + r] * dv[kk], h, l);
      so[(3 * kk + r) * 128 + col] = h;
      so[24 * 128 + (3 * kk + r) * 128 + col] = l;
    }
  }
}

// split-BF16 backward epilogue of one tile (LY_NBN nodes x 3 adjoints) for
// one warp: TMEM lane quarter q (32 neurons of M tile mcol), half `half` of
// each 16-node group.  Group g's activations come from ring buffer n % RING
// (n = j * groups + g, j the CTA's tile count; filled by the activation warp,
// both warps of the quarter read the group's 48 columns); the warp computes
// D = acc * (1 - a^2) of its 8 nodes into its half's staging buffer n & 1;
// the half's warp of quarter 2 stores the buffer (24 rows x 128 neurons, hi
// and lo) with two TMA stores once the half's four warps have written it,
// and releases it when the stores have read it.  Barriers 8 B apart:
// act_full / act_empty [RING], out_full / out_empty [half][buffer].
// Returns false when a wait ran out.
template <int RING>
__device__ __forceinline__ bool bwd_tile_epilogue(uint32_t taddr, long long j, int node0, int mcol, bool active,
                                                  int n_nodes, int half, int q, int lane, const uint8_t* ring,
                                                  uint8_t* outp, uint32_t out_s, uint32_t act_full0,
                                                  uint32_t act_empty0, uint32_t out_full0, uint32_t out_empty0,
                                                  const CUtensorMap* oh, const CUtensorMap* ol,
                                                  volatile int* abort_flag, int* err, long long budget) {
  constexpr int GROUPS = LY_NBN / 16;
  const int col = q * 32 + lane;
#pragma unroll 1
  for (int g = 0; g < GROUPS; ++g) {
    float v[48];
    tmem_ld16(taddr + 48 * g, v);
    tmem_ld16(taddr + 48 * g + 16, v + 16);
    tmem_ld16(taddr + 48 * g + 32, v + 32);
    const long long n = j * GROUPS + g;
    const int b = (int)(n % RING);
    if (!mbar_wait_warp(act_full0 + 8u * b, (uint32_t)((n / RING) & 1), abort_flag, err, budget)) {
      tmem_wait_ld();
      return false;
    }
    const __nv_bfloat16* sa = reinterpret_cast<const __nv_bfloat16*>(ring + (size_t)b * LY_ACT_BYTES);
    __nv_bfloat16 ph[8], pl[8];
    if (half == 0)
      bwd_load_s<0>(sa, col, ph, pl);
    else
      bwd_load_s<1>(sa, col, ph, pl);
    __syncwarp();
    if (lane == 0) mbar_arrive(act_empty0 + 8u * b);
    // staging buffer ob, use u = n >> 1: free once its stores of use u - 1 have read it
    const int ob = (int)(n & 1), slot = 2 * half + ob;
    const uint32_t u = (uint32_t)((n >> 1) & 1);
    if (!mbar_wait_warp(out_empty0 + 8u * slot, u ^ 1u, abort_flag, err, budget)) {
      tmem_wait_ld();
      return false;
    }
    const uint32_t so = out_s + (uint32_t)slot * LY_OUT_BYTES;
    __nv_bfloat16* sop = reinterpret_cast<__nv_bfloat16*>(outp + (size_t)slot * LY_OUT_BYTES);
    tmem_wait_ld();
    if (half == 0)
      bwd_group_s<0>(v, ph, pl, node0 + 16 * g, n_nodes, active, sop, col);
    else
      bwd_group_s<1>(v, ph, pl, node0 + 16 * g, n_nodes, active, sop, col);
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(out_full0 + 8u * slot);
    if (q == 2) {
      if (!mbar_wait_warp(out_full0 + 8u * slot, u, abort_flag, err, budget)) return false;
      if (lane == 0) {
        const int row = (node0 + 16 * g + 8 * half) * 3;
        tma_store_2d(oh, so, mcol * 128, row);
        tma_store_2d(ol, so + LY_OUT_BYTES / 2, mcol * 128, row);
        bulk_commit();
        // the previous group's stores (the other buffer) have read it
        bulk_wait_read<1>();
        if (n >= 1) mbar_arrive(out_empty0 + 8u * (slot ^ 1));
      }
      __syncwarp();
    }
  }
  return true;
}

// split-BF16 forward epilogue of one tile (LY_NF nodes) for one warp: TMEM
// lane quarter q (32 neurons of M tile mcol; this lane's neuron i, active
// when it exists, bias bi), group h of G groups of four warps (one per lane
// quarter) taking chunks h, h + G, ... of 16 nodes.  Per chunk a = tanh(acc
// + b) and, for the last hidden layer (a.dh set), d = 1 - a^2 stored
// directly as BF16 hi + lo; a goes through the group's staging buffer n & 1
// (n the group's chunk count, [16 nodes][128 neurons] hi then lo; nodes past
// the end and neurons past the width staged as zeros), stored by the
// group's quarter-2 warp with two TMA stores at row a.out_row0 + node once
// the group's four warps have written it, released when the stores have
// read it.  Barriers 8 B apart: out_full / out_empty [group][buffer].
// Returns false when a wait ran out.
template <int G>
__device__ __forceinline__ bool fwd_tile_epilogue(uint32_t taddr, long long j, int node0, int mcol, bool active,
                                                  float bi, const LyArgs& a, int h, int q, int lane, uint8_t* outp,
                                                  uint32_t out_s, uint32_t out_full0, uint32_t out_empty0,
                                                  const CUtensorMap* oh, const CUtensorMap* ol,
                                                  volatile int* abort_flag) {
  constexpr int CPG = LY_NF / 16 / G;                 // chunks per group and tile
  constexpr uint32_t BUF = 2u * 16u * 128u * 2u;      // one staging buffer
  const int col = q * 32 + lane, i = mcol * 128 + col;
#pragma unroll 1
  for (int c = 0; c < CPG; ++c) {
    const int ch = h + G * c;
    float v[16];
    tmem_ld16(taddr + 16 * ch, v);
    tmem_wait_ld();
    float av[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) av[k] = v[k] + bi;
    tanh_batch<16>(av);
    if (a.dh) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int node = node0 + 16 * ch + k;
        if (active && node < a.n_nodes) {
          const size_t o = (size_t)node * a.hs + i;
          __nv_bfloat16 dh, dl;
          split_bf(1.0f - av[k] * av[k], dh, dl);
          a.dh[o] = dh;
          a.dl[o] = dl;
        }
      }
    }
    const long long n = j * CPG + c;
    const int slot = 2 * h + (int)(n & 1);
    const uint32_t u = (uint32_t)((n >> 1) & 1);
    if (!mbar_wait_warp(out_empty0 + 8u * slot, u ^ 1u, abort_flag, a.err, a.wait_cycles)) return false;
    const uint32_t so = out_s + (uint32_t)slot * BUF;
    __nv_bfloat16* sop = reinterpret_cast<__nv_bfloat16*>(outp + (size_t)slot * BUF);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      __nv_bfloat16 hv, lv;
      split_bf((active && node0 + 16 * ch + k < a.n_nodes) ? av[k] : 0.0f, hv, lv);
      sop[k * 128 + col] = hv;
      sop[16 * 128 + k * 128 + col] = lv;
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(out_full0 + 8u * slot);
    if (q == 2) {
      if (!mbar_wait_warp(out_full0 + 8u * slot, u, abort_flag, a.err, a.wait_cycles)) return false;
      if (lane == 0) {
        const int row = a.out_row0 + node0 + 16 * ch;
        tma_store_2d(oh, so, mcol * 128, row);
        tma_store_2d(ol, so + BUF / 2, mcol * 128, row);
        bulk_commit();
        bulk_wait_read<1>();  // the group's previous chunk (the other buffer) has been read
        if (n >= 1) mbar_arrive(out_empty0 + 8u * (slot ^ 1));
      }
      __syncwarp();
    }
  }
  return true;
}

// epilogue of the first backward GEMM (last-layer adjoints folded in) for
// one tile (LY_NF nodes; component r0 of the M tile's 128 neurons, this
// lane's neuron i, active when it exists) and one warp: TMEM lane quarter q,
// chunks h, h + G, ... of 16 nodes.  Chunk c's activations a_{L-2} come from
// ring buffer n % RING (n = j * 16 + c, j the CTA's tile count; filled by the
// activation warp); D_{L-2}[node * 3 + r0][i] = acc * (1 - a^2) is stored as
// BF16 hi + lo, or (RTN_FP8, a.y8h set) as e4m3 pieces of D * s8.  Barriers
// 8 B apart: act_full / act_empty [RING].  Returns false when a wait ran out.
template <int RING, int G>
__device__ __forceinline__ bool bw0_tile_epilogue(uint32_t taddr, long long j, int node0, int i, int r0, bool active,
                                                  int h, int q, int lane, const uint8_t* ring, uint32_t act_full0,
                                                  uint32_t act_empty0, const LyArgs& a, volatile int* abort_flag) {
  constexpr int CH = LY_NF / 16;
  const int col = q * 32 + lane;
#pragma unroll 1
  for (int ch = h; ch < CH; ch += G) {
    float v[16];
    tmem_ld16(taddr + 16 * ch, v);
    const long long n = j * CH + ch;
    const int b = (int)(n % RING);
    if (!mbar_wait_warp(act_full0 + 8u * b, (uint32_t)((n / RING) & 1), abort_flag, a.err, a.wait_cycles)) {
      tmem_wait_ld();
      return false;
    }
    const __nv_bfloat16* sa = reinterpret_cast<const __nv_bfloat16*>(ring + (size_t)b * LY_ACT_BYTES);
    __nv_bfloat16 qh[16], ql[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      qh[k] = sa[k * 128 + col];
      ql[k] = sa[16 * 128 + k * 128 + col];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(act_empty0 + 8u * b);
    tmem_wait_ld();
    float dv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float av = __bfloat162float(qh[k]) + __bfloat162float(ql[k]);
      dv[k] = 1.0f - av * av;
    }
    if (a.y8h) {  // RTN_FP8: D * s8 as e4m3 pieces, four nodes per store
      const int tq = lane & 3;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        float d4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) d4[k] = active ? v[4 * m + k] * dv[4 * m + k] * a.s8 : 0.0f;
        store_pieces4(d4, tq, node0 + 16 * ch + 4 * m, a.n_nodes, (size_t)3 * a.hs, (i & ~3) + r0 * a.hs, a.y8h,
                      a.y8m, a.y8l);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int node = node0 + 16 * ch + k;
        if (active && node < a.n_nodes) {
          const size_t o = ((size_t)node * 3 + r0) * a.hs + i;
          __nv_bfloat16 hv, lv;
          split_bf(v[k] * dv[k], hv, lv);
          a.yh[o] = hv;
          a.yl[o] = lv;
        }
      }
    }
  }
  return true;
}

// F8 backward: a_l (= pieces / 448) of the 8 nodes the warp of half H
// stores in the 16-node group starting at node_g, for the lane's row: each
// lane loads the words of rows i & ~3 .. + 3 of one node per piece and quad
// transposes turn them into the lane's row for four nodes (one word per
// piece and four nodes, byte k = node k)
template <int H>
__device__ __forceinline__ void bwd_load8(const LyArgs& a, int node_g, int i, int t, uint32_t (&w)[6]) {
  const int i4 = i & ~3;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const size_t o = (size_t)min(node_g + 8 * H + 4 * m + t, a.n_nodes - 1) * a.hs + i4;
    w[3 * m] = *reinterpret_cast<const uint32_t*>(a.a8h + o);
    w[3 * m + 1] = *reinterpret_cast<const uint32_t*>(a.a8m + o);
    w[3 * m + 2] = *reinterpret_cast<const uint32_t*>(a.a8l + o);
  }
}

// F8 backward epilogue of one 16-node group: D = acc * sc * d, d = 1 - a^2,
// stored as e4m3 pieces of D * s8 (y8, through quad transposes) or as BF16
// hi + lo (yh, yl)
template <int H>
__device__ __forceinline__ void bwd_group8(const float (&v)[48], const uint32_t (&w)[6], int node_g, int i, int t,
                                           bool active, const LyArgs& a) {
  constexpr float inv448 = 1.0f / 448.0f;
  float dv[8];
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    float ah[4], am[4], al[4];
    e4m3x4(quad_transpose(w[3 * m], t), ah);
    e4m3x4(quad_transpose(w[3 * m + 1], t), am);
    e4m3x4(quad_transpose(w[3 * m + 2], t), al);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float av = (ah[k] + am[k] + al[k]) * inv448;
      dv[4 * m + k] = active ? (1.0f - av * av) * a.sc : 0.0f;
    }
  }
  if (a.y8h) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        float d4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) d4[k] = v[3 * (8 * H + 4 * m + k) + r] * dv[4 * m + k] * a.s8;
        // node n = node_g + 8H + 4m + t, row block i & ~3, component r
        const int n0 = node_g + 8 * H + 4 * m;
        store_pieces4(d4, t, n0, a.n_nodes, (size_t)3 * a.hs, (i & ~3) + r * a.hs, a.y8h, a.y8m, a.y8l);
      }
    return;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const int k = 8 * H + kk, node = node_g + k;
    if (active && node < a.n_nodes) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const size_t o = ((size_t)node * 3 + r) * a.hs + i;
        __nv_bfloat16 h, l;
        split_bf(v[3 * k + r] * dv[kk], h, l);
        a.yh[o] = h;
        a.yl[o] = l;
      }
    }
  }
}

// F8 backward: the activations of the tile's first 16-node group (see
// bwd_load8), loaded before the accumulator is ready
__device__ __forceinline__ void bwd8_first(const LyArgs& a, int half, int node0, int ic, int tq, uint32_t (&p8)[6]) {
  if (half == 0)
    bwd_load8<0>(a, node0, ic, tq, p8);
  else
    bwd_load8<1>(a, node0, ic, tq, p8);
}

// F8 backward epilogue of one tile of NODES nodes: each group's activations
// are loaded while the one before it is stored.  The group loop is kept
// rolled: unrolled, the epilogue's code overflows the instruction cache (ncu:
// no_instruction the top stall, 0.79 ms per launch at the precision workload;
// rolled 0.53 ms).
template <int NODES>
__device__ __forceinline__ void bwd8_tile_epilogue(uint32_t taddr, uint32_t (&p8)[6], int node0, int i, int ic,
                                                   int tq, bool active, int half, const LyArgs& a) {
#pragma unroll 1
  for (int g = 0; g < NODES / 16; ++g) {
    float v[48];
    tmem_ld16(taddr + 48 * g, v);
    tmem_ld16(taddr + 48 * g + 16, v + 16);
    tmem_ld16(taddr + 48 * g + 32, v + 32);
    uint32_t n8[6];
    if (g + 1 < NODES / 16) {
      if (half == 0)
        bwd_load8<0>(a, node0 + 16 * (g + 1), ic, tq, n8);
      else
        bwd_load8<1>(a, node0 + 16 * (g + 1), ic, tq, n8);
    }
    tmem_wait_ld();
    if (half == 0)
      bwd_group8<0>(v, p8, node0 + 16 * g, i, tq, active, a);
    else
      bwd_group8<1>(v, p8, node0 + 16 * g, i, tq, active, a);
    if (g + 1 < NODES / 16) {
#pragma unroll
      for (int q8 = 0; q8 < 6; ++q8) p8[q8] = n8[q8];
    }
  }
}

// forward / input epilogue of one 16-node chunk ch of the accumulator, row i:
// a = tanh(acc [* sc] + b) out as BF16 hi + lo (yh, yl), d = 1 - a^2 (dh,
// dl) and, for RTN_FP8, a * 448 as e4m3 pieces (y8)
template <bool F8>
__device__ __forceinline__ void act_chunk_epilogue(uint32_t taddr, int ch, int node0, int i, bool active, float bi,
                                                   int lane, const LyArgs& a) {
  float v[16];
  tmem_ld16(taddr + 16 * ch, v);
  tmem_wait_ld();
  float av[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) av[k] = (F8 ? v[k] * a.sc : v[k]) + bi;
  tanh_batch<16>(av);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int node = node0 + 16 * ch + k;
    if (active && node < a.n_nodes) {
      const size_t o = (size_t)node * a.hs + i;
      __nv_bfloat16 h, l;
      if (a.dh) {
        split_bf(1.0f - av[k] * av[k], h, l);
        a.dh[o] = h;
        a.dl[o] = l;
      }
      if (a.yh) {
        split_bf(av[k], h, l);
        a.yh[o] = h;
        a.yl[o] = l;
      }
    }
  }
  if (a.y8h) {  // RTN_FP8: a * 448 as e4m3 pieces, four nodes per store
    const int tq = lane & 3;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float a4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a4[k] = active ? av[4 * m + k] * 448.0f : 0.0f;
      store_pieces4(a4, tq, node0 + 16 * ch + 4 * m, a.n_nodes, a.hs, i & ~3, a.y8h, a.y8m, a.y8l);
    }
  }
}

// one GEMM layer over all nodes (see the file comment); MODE selects the
// operands' shape and the epilogue
template <int MODE, bool F8 = false>
__global__ void __launch_bounds__(Ly<MODE, F8>::THREADS, 1)
    lay_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ LyMaps bm, LyArgs a) {
  using T = Ly<MODE, F8>;
  constexpr int NS = T::STAGES;
  static_assert(!F8 || MODE == LY_FWD || MODE == LY_BWD, "FP8 hidden GEMMs only");
  constexpr uint32_t B_BYTES = ly_b_bytes<MODE>(), STAGE = ly_stage<MODE, F8>();
  constexpr uint32_t B0 = T::NA * LY_A_BYTES;  // offset of the B tiles in a stage
  extern __shared__ uint8_t smem_raw[];
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t st0 = sraw + pad;
  const uint32_t act_s = st0 + NS * STAGE;  // activation buffers (STAGE_ACT)
  const uint32_t act_bytes = T::STAGE_ACT ? T::ACT_RING * LY_ACT_BYTES : 0;
  const uint32_t out_s = act_s + act_bytes;  // output staging (STAGE_OUT): [group][buffer]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NS * STAGE + act_bytes + T::OUT_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 6 + 2 * T::ACT_RING + T::OUT_BARS);
  static_assert(2 * NS + 6 + 2 * T::ACT_RING + T::OUT_BARS <= 60, "barrier area");
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int k) { return smem_u32(bars + k); };
  auto full_bar = [&](int s) { return bar(s); };
  auto empty_bar = [&](int s) { return bar(NS + s); };
  auto acc_full = [&](int c) { return bar(2 * NS + c); };
  auto tmem_free = [&](int c) { return bar(2 * NS + 2 + c); };
  const uint32_t mma_done = bar(2 * NS + 4);
  const uint32_t stall_bar = bar(2 * NS + 5);  // fault injection: nothing completes it
  auto act_full = [&](int b) { return bar(2 * NS + 6 + b); };
  auto act_empty = [&](int b) { return bar(2 * NS + 6 + T::ACT_RING + b); };
  // staging buffer (group h, buffer b) written by the group's four warps /
  // read out by its TMA stores
  auto out_full = [&](int h, int b) { return bar(2 * NS + 6 + 2 * T::ACT_RING + 2 * h + b); };
  auto out_empty = [&](int h, int b) { return bar(2 * NS + 6 + 2 * T::ACT_RING + 2 * T::OUT_GROUPS + 2 * h + b); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_tiles = (long long)a.n_groups * a.mts;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(acc_full(c), 1);
      mbar_init(tmem_free(c), T::EPI);
    }
    for (int c = 0; c < T::ACT_RING; ++c) {
      mbar_init(act_full(c), 1);
      mbar_init(act_empty(c), T::ACT_READERS);
    }
    for (int c = 0; T::STAGE_OUT && c < 2 * T::OUT_GROUPS; ++c) {
      mbar_init(out_full(c >> 1, c & 1), 4);
      mbar_init(out_empty(c >> 1, c & 1), 1);
    }
    mbar_init(mma_done, 1);
    mbar_init(stall_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(LY_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bm.bh)) : "memory");
    }
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    uint32_t issued = 0, last_ph = 0;
    // fault injection: a bounded wait on a barrier that nothing completes, run
    // out before any copy is issued, so the CTA returns with nothing in flight
    if (a.stall) ok = mbar_wait_warp(stall_bar, 0, abort_flag, a.err, a.wait_cycles);
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int grp = (int)(t / a.mts), mt = (int)(t % a.mts);
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err, a.wait_cycles))) break;
        if (elect_one()) {
          const uint32_t sa = st0 + s * STAGE;
          mbar_expect_tx(full_bar(s), STAGE);
          tma_load_2d(sa, &amap, kb * T::KB, a.a_row0 + mt * 128, full_bar(s));
          if (T::NA == 2)
            tma_load_2d(sa + LY_A_BYTES, &amap, kb * T::KB, a.a_row0 + a.a_lo + mt * 128, full_bar(s));
          tma_load_2d(sa + B0, &bm.bh, kb * T::KB, a.b_row0 + grp * T::N, full_bar(s));
          tma_load_2d(sa + B0 + B_BYTES, &bm.bl, kb * T::KB, a.b_row0 + grp * T::N, full_bar(s));
          if (F8) tma_load_2d(sa + B0 + 2 * B_BYTES, &bm.b3, kb * T::KB, a.b_row0 + grp * T::N, full_bar(s));
        }
        __syncwarp();
        issued |= 1u << s;
        last_ph = (last_ph & ~(1u << s)) | (ph << s);
        if (++s == NS) { s = 0; ph ^= 1u; }
      }
    }
    for (int q = 0; q < NS; ++q)
      if (issued & (1u << q)) {
        const long long t0 = clock64();
        while (!mbar_try(full_bar(q), (last_ph >> q) & 1u) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = F8 ? idesc_e4m3(128, T::N) : idesc_bf16(128, T::N);  // both operands K-major
    int s = 0, acc = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      if (!(ok = mbar_wait_warp(tmem_free(acc), aph ^ 1u, abort_flag, a.err, a.wait_cycles))) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * 256u;
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err, a.wait_cycles))) break;
        tc_fence_after();
        const uint32_t sa = st0 + s * STAGE;
        // two K steps per 64 B row: 16 BF16 or 32 e4m3 elements each
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ah = kmajor_desc(sa + ks * 32u, LY_SBO, LY_SWZ);
          const uint64_t bh = kmajor_desc(sa + B0 + ks * 32u, LY_SBO, LY_SWZ);
          const uint64_t bl = kmajor_desc(sa + B0 + B_BYTES + ks * 32u, LY_SBO, LY_SWZ);
          if constexpr (F8) {
            const uint64_t b3 = kmajor_desc(sa + B0 + 2 * B_BYTES + ks * 32u, LY_SBO, LY_SWZ);
            mma_f8_elect(d, ah, bh, idesc, (kb | ks) != 0);
            mma_f8_elect(d, ah, bl, idesc, 1u);
            mma_f8_elect(d, ah, b3, idesc, 1u);
          } else {
            mma_bf16_elect(d, ah, bh, idesc, (kb | ks) != 0);
            mma_bf16_elect(d, ah, bl, idesc, 1u);
            if (T::NA == 2) mma_bf16_elect(d, kmajor_desc(sa + LY_A_BYTES + ks * 32u, LY_SBO, LY_SWZ), bh, idesc, 1u);
          }
        }
        mma_commit_elect(empty_bar(s));
        if (++s == NS) { s = 0; ph ^= 1u; }
      }
      if (!ok) break;
      mma_commit_elect(acc_full(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    mma_commit_elect(mma_done);
    const long long t0 = clock64();
    while (!mbar_try(mma_done, 0) && clock64() - t0 < WAIT_CYCLES) {
    }
  } else if (T::STAGE_ACT && warp == 2 + T::EPI) {
    // ---------------- activation loader (split-BF16 backward GEMMs): chunk
    // c of every tile (16 nodes x 128 neurons, hi and lo) into ring buffer
    // n % ACT_RING (n the CTA's chunk count) once the epilogue has released
    // the buffer's previous chunk
    if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bm.sh)) : "memory");
    bool ok = true;
    uint32_t issued = 0, last_ph = 0;
    long long n = 0;
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int grp = (int)(t / a.mts), mt = (int)(t % a.mts);
      const int mc = MODE == LY_BW0 ? mt % a.mtpr : mt;  // neuron block (BW0: of component r)
      for (int c = 0; c < T::ACT_CHUNKS; ++c, ++n) {
        const int b = (int)(n % T::ACT_RING);
        const uint32_t ph = (uint32_t)((n / T::ACT_RING) & 1);
        if (!(ok = mbar_wait_warp(act_empty(b), ph ^ 1u, abort_flag, a.err, a.wait_cycles))) break;
        if (elect_one()) {
          const uint32_t dst = act_s + (uint32_t)b * LY_ACT_BYTES;
          const int row = a.act_row0 + grp * T::NODES + 16 * c;
          mbar_expect_tx(act_full(b), LY_ACT_BYTES);
          tma_load_2d(dst, &bm.sh, mc * 128, row, act_full(b));
          tma_load_2d(dst + LY_ACT_BYTES / 2, &bm.sl, mc * 128, row, act_full(b));
        }
        __syncwarp();
        issued |= 1u << b;
        last_ph = (last_ph & ~(1u << b)) | (ph << b);
      }
    }
    // the ring's last copies have landed before the CTA may exit
    for (int b = 0; b < T::ACT_RING; ++b)
      if (issued & (1u << b)) {
        const long long t0 = clock64();
        while (!mbar_try(act_full(b), (last_ph >> b) & 1u) && clock64() - t0 < a.wait_cycles) {
        }
      }
  } else if (warp < 2 + T::EPI) {
    // ---------------- epilogue: TMEM lane quarter warp % 4, one output row
    // per lane; the two warps of a quarter take alternate 16-column chunks.
    // Each chunk issues its loads first and predicates only the stores, so
    // the loads and the activation arithmetic of 16 columns overlap.
    const int q = warp & 3, half = (warp - 2) >> 2;
    int acc = 0;
    uint32_t aph = 0;
    long long j = 0;  // the CTA's tile count (activation buffer j % 2)
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
      const int grp = (int)(t / a.mts), mt = (int)(t % a.mts);
      // output row i (BW0: row k of component r)
      const int r0 = MODE == LY_BW0 ? mt / a.mtpr : 0;
      const int i = (MODE == LY_BW0 ? mt % a.mtpr : mt) * 128 + q * 32 + lane;
      const bool active = i < a.m_rows;
      const int ic = active ? i : 0;  // a row that exists, for the loads
      const int node0 = grp * T::NODES;
      const float bi = T::ACT ? __ldg(a.bias + ic) : 0.0f;
      // F8 backward: the first group's activations are loaded while the
      // accumulator is still being computed, each later group's while the
      // one before it is stored
      uint32_t p8[6];
      const int tq = lane & 3;
      if (MODE == LY_BWD && F8) bwd8_first(a, half, node0, ic, tq, p8);
      if (!mbar_wait_warp(acc_full(acc), aph, abort_flag, a.err, a.wait_cycles)) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * 256u;
      if (MODE == LY_BWD && F8) bwd8_tile_epilogue<T::NODES>(taddr, p8, node0, i, ic, tq, active, half, a);
      if (MODE == LY_BWD && !F8) {
        if (!bwd_tile_epilogue<T::ACT_RING>(taddr, j, node0, mt, active, a.n_nodes, half, q, lane,
                                            sm + NS * STAGE, sm + (out_s - st0), out_s, act_full(0), act_empty(0),
                                            out_full(0, 0), out_empty(0, 0), &bm.oh, &bm.ol, abort_flag, a.err,
                                            a.wait_cycles))
          break;
      }
      if (MODE == LY_FWD && !F8) {
        if (!fwd_tile_epilogue<T::OUT_GROUPS>(taddr, j, node0, mt, active, bi, a, half, q, lane, sm + (out_s - st0),
                                              out_s, out_full(0, 0), out_empty(0, 0), &bm.oh, &bm.ol, abort_flag))
          break;
      }
      if (MODE == LY_BW0) {
        if (!bw0_tile_epilogue<T::ACT_RING, T::EPI / 4>(taddr, j, node0, i, r0, active, half, q, lane,
                                                         sm + NS * STAGE, act_full(0), act_empty(0), a, abort_flag))
          break;
      }
      for (int ch = half; MODE != LY_BWD && MODE != LY_BW0 && !(MODE == LY_FWD && !F8) && ch < T::N / 16;
           ch += T::EPI / 4) {
        if (T::ACT) {
          act_chunk_epilogue<F8>(taddr, ch, node0, i, active, bi, lane, a);
        } else {
          float v[16];
          tmem_ld16(taddr + 16 * ch, v);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int c = 16 * ch + k, node = node0 + c / 3, r = c % 3;
            if (active && node < a.n_nodes) a.JD[((size_t)node * 3 + r) * NZ + i] = v[k];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    // the staged stores have completed before the CTA's shared memory goes
    if (T::STAGE_OUT && lane == 0 && (warp & 3) == 2) bulk_wait_all();
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LY_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- CTA pairs
// The backward and forward hidden GEMMs (split BF16 and F8) on CTA pairs
// (cta_group::2): one pair tile is M = 256 neurons (128 per CTA, its own
// weight rows) x N (backward 240 = 80 nodes x 3 adjoints, forward 256 nodes;
// each CTA loads N / 2 rows of every B piece, which the MMA reads across the
// pair) x K.  Each CTA's tensor memory holds its 128 rows x N columns, so the
// epilogues are the single-CTA ones (split BF16: activation ring and staged
// TMA stores; F8: direct loads and piece stores).  Every B
// row of a node group is read by two pair tiles instead of four M tiles:
// per SM 23-24 KB instead of 38-40 KB per K block, the traffic through L2
// that bounds the single-CTA kernels.  Rank 0 issues the MMAs; both CTAs'
// TMA loads complete on rank 0's stage barriers and both release their
// stages on the MMAs' multicast commits; both CTAs' epilogues free an
// accumulator on rank 0's barrier.  (The first backward GEMM on pairs
// measured slower, 0.602 vs 0.592 ms per launch: its epilogue bounds it.)
constexpr int LB2_STAGES = 6;
constexpr int LB2_RING = 3;  // backward: activation ring buffers
template <int MODE, bool F8 = false>
struct Lb2 {
  using T = Ly<MODE, F8>;
  static_assert(T::NA == 1, "one weight tile per stage");
  static constexpr bool RING = MODE == LY_BWD && !F8;                 // activation loader warp + ring
  static constexpr int N_RING = RING ? LB2_RING : 0;
  static constexpr uint32_t B_BYTES = (uint32_t)(T::N / 2) * 64u;     // one CTA's half of a B piece
  static constexpr uint32_t B0 = LY_A_BYTES;                          // B's offset in a stage
  static constexpr uint32_t LOAD = B0 + (uint32_t)T::NB * B_BYTES;    // bytes one CTA loads per stage
  static constexpr uint32_t STAGE = (LOAD + 1023u) / 1024u * 1024u;   // 1 KB aligned stages
  static constexpr uint32_t RING_BYTES = (uint32_t)N_RING * LY_ACT_BYTES;
  static constexpr int THREADS = 64 + 32 * T::EPI + (RING ? 32 : 0);  // TMA, MMA, epilogue, [loader]
  static constexpr size_t SMEM = LB2_STAGES * STAGE + RING_BYTES + T::OUT_BYTES + 1024 + 512;
};
static_assert(Lb2<LY_BWD>::SMEM <= 232448 && Lb2<LY_FWD>::SMEM <= 232448 && Lb2<LY_BWD, true>::SMEM <= 232448 &&
                  Lb2<LY_FWD, true>::SMEM <= 232448,
              "shared memory");
static_assert(Lb2<LY_BWD>::B_BYTES % 512 == 0 && Lb2<LY_FWD>::B_BYTES % 512 == 0 && Lb2<LY_BWD, true>::STAGE % 1024 == 0,
              "swizzle atoms");

// bounded wait with cluster-scope acquire (barriers with arrivals from the
// peer CTA), every lane of a warp, warp-uniform result
__device__ __forceinline__ bool wait_cl_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                             long long budget) {
  bool ok = mbar_try_cl(bar, parity);
  if (!ok) {
    const long long t0 = clock64();
    for (;;) {
      if (mbar_try_cl_sleep(bar, parity, WAIT_SLEEP_NS)) {
        ok = true;
        break;
      }
      if (*abort_flag) break;
      if (clock64() - t0 > budget) {
        *abort_flag = 1;
        atomicExch(err, (int)RTN_E_TIMEOUT);
        break;
      }
    }
  }
  return __all_sync(0xffffffffu, ok);
}

template <int MODE, bool F8 = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Lb2<MODE, F8>::THREADS, 1)
    lay2_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ LyMaps bm, LyArgs a) {
  using T = Ly<MODE, F8>;
  using P = Lb2<MODE, F8>;
  constexpr int NS = LB2_STAGES, NR = P::N_RING;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t st0 = sraw + pad;
  const uint32_t ring_s = st0 + NS * P::STAGE;
  const uint32_t out_s = ring_s + P::RING_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (out_s - st0) + T::OUT_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 6 + 2 * NR + T::OUT_BARS);
  static_assert(2 * NS + 6 + 2 * NR + T::OUT_BARS <= 60, "barrier area");
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int k) { return smem_u32(bars + k); };
  auto full_bar = [&](int s) { return bar(s); };
  auto empty_bar = [&](int s) { return bar(NS + s); };
  auto acc_full = [&](int c) { return bar(2 * NS + c); };
  auto tmem_free = [&](int c) { return bar(2 * NS + 2 + c); };
  const uint32_t mma_done = bar(2 * NS + 4);
  const uint32_t stall_bar = bar(2 * NS + 5);  // fault injection: nothing completes it
  auto act_full = [&](int b) { return bar(2 * NS + 6 + b); };
  auto act_empty = [&](int b) { return bar(2 * NS + 6 + NR + b); };
  const uint32_t out_full0 = bar(2 * NS + 6 + 2 * NR), out_empty0 = bar(2 * NS + 6 + 2 * NR + 2 * T::OUT_GROUPS);

  const uint32_t rank = cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
  const int mps = a.mts >> 1;  // pair tiles per node group
  const long long n_tiles = (long long)a.n_groups * mps;
  const long long budget = a.wait_cycles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(acc_full(c), 1);
      mbar_init(tmem_free(c), 2 * T::EPI);
    }
    mbar_init(mma_done, 1);
    mbar_init(stall_bar, 1);
    for (int c = 0; c < NR; ++c) {
      mbar_init(act_full(c), 1);
      mbar_init(act_empty(c), T::ACT_READERS);
    }
    for (int c = 0; T::STAGE_OUT && c < 2 * T::OUT_GROUPS; ++c) {
      mbar_init(out_full0 + 8u * c, 4);
      mbar_init(out_empty0 + 8u * c, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(LY_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // both CTAs must address the same tensor-memory columns
  if (threadIdx.x == 0 && rank == 1) {
    uint32_t other;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(mapa(smem_u32(tmem_slot), 0)) : "memory");
    if (other != tmem) {
      atomicExch(a.err, (int)RTN_E_UNSUPPORTED);
      *abort_flag = 1;
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(mapa(smem_u32((const void*)abort_flag), 0)), "r"(1)
                   : "memory");
    }
  }
  cluster_sync();
  const bool run = *abort_flag == 0;

  if (run && warp == 0) {
    // ---------------- TMA producer (both CTAs): this CTA's 128 weight rows
    // and its N / 2 rows of B (hi, lo) of every K block, onto rank 0's stage
    // barrier
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bm.bh)) : "memory");
    }
    const uint32_t full0 = mapa(full_bar(0), 0);
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    // fault injection: a bounded wait on a barrier that nothing completes, run
    // out before any copy is issued
    if (a.stall) ok = mbar_wait_warp(stall_bar, 0, abort_flag, a.err, budget);
    for (long long t = pair; t < n_tiles && ok; t += n_pairs) {
      const int grp = (int)(t / mps), mp = (int)(t % mps);
      const int arow = a.a_row0 + (mp * 2 + (int)rank) * 128;
      const int brow = a.b_row0 + grp * T::N + (int)rank * (T::N / 2);
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = wait_cl_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err, budget))) break;
        if (elect_one()) {
          const uint32_t sa = st0 + s * P::STAGE, fb = full0 + 8u * s;
          if (rank == 0) mbar_expect_tx(full_bar(s), 2u * P::LOAD);
          tma_load_2d_pair(sa, &amap, kb * T::KB, arow, fb);
          tma_load_2d_pair(sa + P::B0, &bm.bh, kb * T::KB, brow, fb);
          tma_load_2d_pair(sa + P::B0 + P::B_BYTES, &bm.bl, kb * T::KB, brow, fb);
          if (F8) tma_load_2d_pair(sa + P::B0 + 2 * P::B_BYTES, &bm.b3, kb * T::KB, brow, fb);
        }
        __syncwarp();
        if (++s == NS) { s = 0; ph ^= 1u; }
      }
    }
    // tail: every stage released, so no copy or commit lands after exit
    for (int i = 0; i < NS && ok; ++i) {
      ok = wait_cl_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err, budget);
      if (++s == NS) { s = 0; ph ^= 1u; }
    }
  } else if (run && warp == 1 && rank == 0) {
    // ---------------- MMA issuer of the pair: two K steps per 64 B row
    // against B's pieces (hi, lo; F8 hi, mid, lo), M = 256
    constexpr uint32_t idesc = F8 ? idesc_e4m3(256, T::N) : idesc_bf16(256, T::N);
    int s = 0, acc = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (long long t = pair; t < n_tiles && ok; t += n_pairs) {
      if (!(ok = wait_cl_warp(tmem_free(acc), aph ^ 1u, abort_flag, a.err, budget))) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * 256u;
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err, budget))) break;
        tc_fence_after();
        const uint32_t sa = st0 + s * P::STAGE;
        if constexpr (F8) {
          uint64_t ad[2], bd[6];
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            ad[ks] = kmajor_desc(sa + ks * 32u, LY_SBO, LY_SWZ);
#pragma unroll
            for (int pc = 0; pc < 3; ++pc)
              bd[3 * ks + pc] = kmajor_desc(sa + P::B0 + pc * P::B_BYTES + ks * 32u, LY_SBO, LY_SWZ);
          }
          mma2_f8_x6(d, ad, bd, idesc, kb != 0);
        } else {
          uint64_t ad[4], bd[4];
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t aw = kmajor_desc(sa + ks * 32u, LY_SBO, LY_SWZ);
            ad[2 * ks] = aw;
            ad[2 * ks + 1] = aw;
            bd[2 * ks] = kmajor_desc(sa + P::B0 + ks * 32u, LY_SBO, LY_SWZ);
            bd[2 * ks + 1] = kmajor_desc(sa + P::B0 + P::B_BYTES + ks * 32u, LY_SBO, LY_SWZ);
          }
          mma2_bf16_x4(d, ad, bd, idesc, kb != 0);
        }
        commit2(empty_bar(s), 3);
        if (++s == NS) { s = 0; ph ^= 1u; }
      }
      if (!ok) break;
      commit2(acc_full(acc), 3);
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    commit2(mma_done, 3);
    const long long t0 = clock64();
    while (!mbar_try(mma_done, 0) && clock64() - t0 < budget) {
    }
  } else if (run && P::RING && warp == 2 + T::EPI) {
    // ---------------- activation loader (backward, both CTAs): chunk c of
    // every tile (16 nodes x this CTA's 128 neurons, hi and lo) into ring
    // buffer n % LB2_RING once the epilogue has released it
    if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bm.sh)) : "memory");
    bool ok = true;
    uint32_t issued = 0, last_ph = 0;
    long long n = 0;
    for (long long t = pair; t < n_tiles && ok; t += n_pairs) {
      const int grp = (int)(t / mps), mc = (int)(t % mps) * 2 + (int)rank;
      for (int c = 0; c < T::ACT_CHUNKS; ++c, ++n) {
        constexpr int NRD = NR > 0 ? NR : 1;  // (no ring in the forward GEMM)
        const int b = (int)(n % NRD);
        const uint32_t ph = (uint32_t)((n / NRD) & 1);
        if (!(ok = mbar_wait_warp(act_empty(b), ph ^ 1u, abort_flag, a.err, budget))) break;
        if (elect_one()) {
          const uint32_t dst = ring_s + (uint32_t)b * LY_ACT_BYTES;
          const int row = a.act_row0 + grp * T::NODES + 16 * c;
          mbar_expect_tx(act_full(b), LY_ACT_BYTES);
          tma_load_2d(dst, &bm.sh, mc * 128, row, act_full(b));
          tma_load_2d(dst + LY_ACT_BYTES / 2, &bm.sl, mc * 128, row, act_full(b));
        }
        __syncwarp();
        issued |= 1u << b;
        last_ph = (last_ph & ~(1u << b)) | (ph << b);
      }
    }
    // the ring's last copies have landed before the CTA may exit
    for (int b = 0; b < NR; ++b)
      if (issued & (1u << b)) {
        const long long t0 = clock64();
        while (!mbar_try(act_full(b), (last_ph >> b) & 1u) && clock64() - t0 < budget) {
        }
      }
  } else if (run && warp >= 2 && warp < 2 + T::EPI) {
    // ---------------- epilogue (both CTAs): this CTA's 128 rows, as the
    // single-CTA epilogue
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t tfree0 = mapa(tmem_free(0), 0);
    int acc = 0;
    uint32_t aph = 0;
    long long j = 0;
    for (long long t = pair; t < n_tiles; t += n_pairs, ++j) {
      const int grp = (int)(t / mps), mc = (int)(t % mps) * 2 + (int)rank;
      const int i = mc * 128 + q * 32 + lane;
      const bool active = i < a.m_rows;
      const float bi = MODE == LY_FWD ? __ldg(a.bias + (active ? i : 0)) : 0.0f;
      uint32_t p8[6];
      const int tq = lane & 3;
      if constexpr (MODE == LY_BWD && F8) bwd8_first(a, half, grp * T::NODES, active ? i : 0, tq, p8);
      if (!wait_cl_warp(acc_full(acc), aph, abort_flag, a.err, budget)) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * 256u;
      bool ok = true;
      if constexpr (MODE == LY_BWD && F8)
        bwd8_tile_epilogue<T::NODES>(taddr, p8, grp * T::NODES, i, active ? i : 0, tq, active, half, a);
      else if constexpr (MODE == LY_FWD && F8)
        for (int ch = half; ch < T::N / 16; ch += T::EPI / 4)
          act_chunk_epilogue<true>(taddr, ch, grp * T::NODES, i, active, bi, lane, a);
      else if constexpr (MODE == LY_BWD)
        ok = bwd_tile_epilogue<LB2_RING>(taddr, j, grp * T::NODES, mc, active, a.n_nodes, half, q, lane,
                                         sm + (ring_s - st0), sm + (out_s - st0), out_s, act_full(0), act_empty(0),
                                         out_full0, out_empty0, &bm.oh, &bm.ol, abort_flag, a.err, budget);
      else
        ok = fwd_tile_epilogue<T::OUT_GROUPS>(taddr, j, grp * T::NODES, mc, active, bi, a, half, q, lane,
                                              sm + (out_s - st0), out_s, out_full0, out_empty0, &bm.oh, &bm.ol,
                                              abort_flag);
      if (!ok) break;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_cluster(tfree0 + 8u * acc);
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    // the staged stores have completed before the CTA's shared memory goes
    if (T::STAGE_OUT && lane == 0 && q == 2) bulk_wait_all();
  }

  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LY_TMEM_COLS)
                 : "memory");
  }
}
// node inputs z = [x; u] as the K-major B operand of the input-layer GEMM:
// [node][32] BF16 hi + lo (columns 17..31 stay zero)
__global__ void __launch_bounds__(256) lay_z_kernel(const float* __restrict__ x, const float* __restrict__ u,
                                                    const int* __restrict__ node_inst, int n_nodes,
                                                    __nv_bfloat16* __restrict__ zh, __nv_bfloat16* __restrict__ zl) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n_nodes * NZ) return;
  const int n = (int)(e / NZ), j = (int)(e % NZ);
  const float v = j < NX ? x[(size_t)(n + node_inst[n]) * NX + j] : u[(size_t)n * NU + (j - NX)];
  __nv_bfloat16 h, l;
  split_bf(v, h, l);
  zh[(size_t)n * LY_KB + j] = h;
  zl[(size_t)n * LY_KB + j] = l;
}

// output layer f_D = W_L a_L + b_L (warp per node) and the last layer's
// adjoints D_L[node * 3 + r][i] = d_L[i] W_L[r][i] (split hi + lo), for a
// network with no hidden -> hidden layer or a last width that is not a
// multiple of 8
__global__ void __launch_bounds__(256) lay_out_kernel(const float* __restrict__ WL, const float* __restrict__ bL,
                                                      int h, int n_nodes, int hs, const __nv_bfloat16* __restrict__ xh,
                                                      const __nv_bfloat16* __restrict__ xl, float* __restrict__ fD,
                                                      __nv_bfloat16* __restrict__ Dh, __nv_bfloat16* __restrict__ Dl,
                                                      int HP) {
  const int lane = threadIdx.x & 31;
  for (long long node = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; node < n_nodes;
       node += ((long long)gridDim.x * blockDim.x) >> 5) {
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    const size_t row = (size_t)node * hs;
    // four columns per lane per step, loads first
    for (int i0 = lane; i0 < h; i0 += 128) {
      float av[4], dv[4], w0[4], w1[4], w2[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = min(i0 + 32 * t, h - 1);
        av[t] = __bfloat162float(xh[row + i]) + __bfloat162float(xl[row + i]);
        dv[t] = 1.0f - av[t] * av[t];
        w0[t] = __ldg(WL + i);
        w1[t] = __ldg(WL + HP + i);
        w2[t] = __ldg(WL + 2 * HP + i);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = i0 + 32 * t;
        if (i >= h) break;
        f0 = fmaf(w0[t], av[t], f0);
        f1 = fmaf(w1[t], av[t], f1);
        f2 = fmaf(w2[t], av[t], f2);
        if (!Dh) continue;  // the adjoints are folded into the first backward GEMM
        __nv_bfloat16 hh, ll;
        const size_t o = (size_t)node * 3 * hs + i;
        split_bf(dv[t] * w0[t], hh, ll);
        Dh[o] = hh;
        Dl[o] = ll;
        split_bf(dv[t] * w1[t], hh, ll);
        Dh[o + hs] = hh;
        Dl[o + hs] = ll;
        split_bf(dv[t] * w2[t], hh, ll);
        Dh[o + 2 * hs] = hh;
        Dl[o + 2 * hs] = ll;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f0 += __shfl_xor_sync(0xffffffffu, f0, o);
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    }
    if (lane == 0) {
      fD[node * NO + 0] = f0 + bL[0];
      fD[node * NO + 1] = f1 + bL[1];
      fD[node * NO + 2] = f2 + bL[2];
    }
  }
}

// output layer f_D = W_L a_L + b_L with no adjoints (h <= 512, h % 8 == 0):
// a warp per node, each lane reading 8 consecutive neurons of a_L hi and lo
// as one 16 B load each, both steps' loads issued before the arithmetic
__global__ void __launch_bounds__(256) lay_fd_kernel(const float* __restrict__ WL, const float* __restrict__ bL,
                                                     int h, int n_nodes, int hs,
                                                     const __nv_bfloat16* __restrict__ xh,
                                                     const __nv_bfloat16* __restrict__ xl, float* __restrict__ fD,
                                                     int HP) {
  const int lane = threadIdx.x & 31;
  for (long long node = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; node < n_nodes;
       node += ((long long)gridDim.x * blockDim.x) >> 5) {
    const size_t row = (size_t)node * hs;
    uint4 ph[2], pl[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = lane * 8 + 256 * k;
      if (c < h) {
        ph[k] = __ldg(reinterpret_cast<const uint4*>(xh + row + c));
        pl[k] = __ldg(reinterpret_cast<const uint4*>(xl + row + c));
      }
    }
    float f[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = lane * 8 + 256 * k;
      if (c >= h) break;
      const __nv_bfloat16* eh = reinterpret_cast<const __nv_bfloat16*>(&ph[k]);
      const __nv_bfloat16* el = reinterpret_cast<const __nv_bfloat16*>(&pl[k]);
      float av[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) av[t] = __bfloat162float(eh[t]) + __bfloat162float(el[t]);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float4 w0 = __ldg(reinterpret_cast<const float4*>(WL + (size_t)r * HP + c));
        const float4 w1 = __ldg(reinterpret_cast<const float4*>(WL + (size_t)r * HP + c + 4));
        float v = f[r];
        v = fmaf(w0.x, av[0], v);
        v = fmaf(w0.y, av[1], v);
        v = fmaf(w0.z, av[2], v);
        v = fmaf(w0.w, av[3], v);
        v = fmaf(w1.x, av[4], v);
        v = fmaf(w1.y, av[5], v);
        v = fmaf(w1.z, av[6], v);
        v = fmaf(w1.w, av[7], v);
        f[r] = v;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < 3; ++r) f[r] += __shfl_xor_sync(0xffffffffu, f[r], o);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < 3; ++r) fD[node * NO + r] = f[r] + bL[r];
  }
}

}  // namespace

float quantize_e4m3(float* w, size_t n) {
  float amax = 0.0f;
  for (size_t i = 0; i < n; ++i) amax = std::max(amax, std::fabs(w[i]));
  if (!(amax > 0.0f)) return 1.0f;
  const float sc = amax / 448.0f;
  for (size_t i = 0; i < n; ++i) {
    const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(w[i] / sc, __NV_SATFINITE, __NV_E4M3);
    w[i] = sc * __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
  }
  return sc;
}

const void* mlp_lay_fn() { return reinterpret_cast<const void*>(&lay_kernel<LY_FWD>); }
size_t mlp_lay_smem() { return std::max(std::max(ly_smem<LY_JD>(), ly_smem<LY_BW0>()), ly_smem<LY_IN>()); }

cudaError_t mlp_lay_prepare(rtn_ctx* ctx, std::string& err) {
  TcNet& tc = ctx->net.tc;
  if (tc.lay) return cudaSuccess;
  Net& net = ctx->net;
  const int L = net.n_layers, n = ctx->lay.n_nodes, HP = tc.h_pad;
  const long long npad = ((long long)n + LY_NODE_PAD - 1) / LY_NODE_PAD * LY_NODE_PAD;
  if (3 * npad >= (1LL << 31) || (long long)(L - 1) * npad >= (1LL << 31)) {
    err = "layered reverse mode: more nodes than the 32-bit tensor coordinates address";
    return cudaSuccess;
  }
  LayState* s = new (std::nothrow) LayState();
  if (!s) return cudaErrorMemoryAllocation;
  tc.lay = s;
  cudaError_t es = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  if (es == cudaSuccess) es = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
  if (es == cudaSuccess) es = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
  if (es != cudaSuccess) return es;
  s->hs = HP;
  s->npad = (int)npad;
  s->fp8 = ctx->opt.precision == RTN_FP8;
  cudaError_t e;
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p) {
      if ((e = cudaMalloc(&s->xb[b][p], (size_t)3 * npad * HP * 2)) != cudaSuccess) return e;
      if ((e = cudaMemset(s->xb[b][p], 0, (size_t)3 * npad * HP * 2)) != cudaSuccess) return e;
    }
  for (int p = 0; p < 2; ++p) {
    const size_t bytes = (size_t)(L - 1) * npad * HP * 2;
    if ((e = cudaMalloc(&s->act[p], bytes)) != cudaSuccess) return e;
    if ((e = cudaMemset(s->act[p], 0, bytes)) != cudaSuccess) return e;
  }
  for (int p = 0; p < 2; ++p) {
    if ((e = cudaMalloc(&s->z[p], (size_t)npad * LY_KB * 2)) != cudaSuccess) return e;
    if ((e = cudaMemset(s->z[p], 0, (size_t)npad * LY_KB * 2)) != cudaSuccess) return e;
  }
  {
    // W_0 rows (FP32 [17][HP] transposed in the tensor-core pack) split hi + lo
    std::vector<float> W0((size_t)NZ * HP);
    if ((e = cudaMemcpy(W0.data(), tc.W0, W0.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
    std::vector<__nv_bfloat16> w((size_t)2 * HP * LY_KB, __float2bfloat16_rn(0.0f));
    for (int i = 0; i < HP; ++i)
      for (int j = 0; j < NZ; ++j) {
        const float v = W0[(size_t)j * HP + i];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        w[(size_t)i * LY_KB + j] = h;
        w[(size_t)(HP + i) * LY_KB + j] = __float2bfloat16_rn(v - __bfloat162float(h));
      }
    if ((e = cudaMalloc(&s->w0s, w.size() * 2)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(s->w0s, w.data(), w.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  const int nh = L - 2;
  if (nh >= 1) {
    for (int p = 0; p < 2; ++p) {
      if ((e = cudaMalloc(&s->dd[p], (size_t)npad * HP * 2)) != cudaSuccess) return e;
      if ((e = cudaMemset(s->dd[p], 0, (size_t)npad * HP * 2)) != cudaSuccess) return e;
    }
    // M_r[k][i] = W_{L-2}[i][k] W_L[r][i] with the BF16-rounded hidden
    // weights of the other shapes and the FP32 output layer, split hi + lo
    const int hk = net.widths[L - 2], hi_ = net.widths[L - 1];
    std::vector<float> Wa((size_t)hi_ * hk), Wl((size_t)NO * hi_);
    if ((e = cudaMemcpy(Wa.data(), net.W32 + net.w_off[L - 2], Wa.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpy(Wl.data(), net.W32 + net.w_off[L - 1], Wl.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    std::vector<__nv_bfloat16> M((size_t)6 * HP * HP, __float2bfloat16_rn(0.0f));
    for (int r = 0; r < NO; ++r)
      for (int k = 0; k < hk; ++k)
        for (int i = 0; i < hi_; ++i) {
          // the hidden weight as the other BF16 GEMMs see it (RTN_FP8: the
          // dequantised weight itself)
          const float wa = s->fp8 ? Wa[(size_t)i * hk + k] : __bfloat162float(__float2bfloat16_rn(Wa[(size_t)i * hk + k]));
          const float m = wa * Wl[(size_t)r * hi_ + i];
          const __nv_bfloat16 h = __float2bfloat16_rn(m);
          M[((size_t)r * HP + k) * HP + i] = h;
          M[((size_t)(3 + r) * HP + k) * HP + i] = __float2bfloat16_rn(m - __bfloat162float(h));
        }
    if ((e = cudaMalloc(&s->mw, M.size() * 2)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(s->mw, M.data(), M.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }

  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || !fn || qr != cudaDriverEntryPointSuccess) {
    err = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint32_t estr[2] = {1, 1};
  auto enc_k = [&](void* mp, void* ptr, int inner, long long rows, int box_rows) -> bool {
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t str[1] = {(cuuint64_t)inner * 2};
    const cuuint32_t box[2] = {(cuuint32_t)LY_KB, (cuuint32_t)box_rows};
    return encode(reinterpret_cast<CUtensorMap*>(mp), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, str, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  auto enc = [&](void* mp, void* ptr, long long rows, int box_rows) { return enc_k(mp, ptr, HP, rows, box_rows); };
  if (!enc_k(s->mw0, s->w0s, LY_KB, 2LL * HP, 128) || !enc_k(s->mz[0], s->z[0], LY_KB, npad, LY_NF) ||
      !enc_k(s->mz[1], s->z[1], LY_KB, npad, LY_NF)) {
    err = "cuTensorMapEncodeTiled failed";
    return cudaSuccess;
  }
  if ((e = cudaFuncSetAttribute(lay_kernel<LY_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ly_smem<LY_IN>())) != cudaSuccess)
    return e;

  // maps: forward tiles read the stacked activations (box 256 rows),
  // backward and Jacobian tiles read adjoints (box 240 rows); no box reaches
  // past its layer (rows padded to a multiple of both tiles)
  for (int p = 0; p < 2; ++p)
    if (!enc(s->ma[p], s->act[p], (long long)(L - 1) * npad, LY_NF) ||
        !enc(s->ma2[p], s->act[p], (long long)(L - 1) * npad, LY_NF / 2)) {
      err = "cuTensorMapEncodeTiled failed";
      return cudaSuccess;
    }
  // the backward epilogues' activation blocks: 128 neurons x LY_NBN nodes,
  // unswizzled (a lane reads its neuron's column)
  for (int p = 0; p < 2; ++p) {
    const cuuint64_t dims[2] = {(cuuint64_t)HP, (cuuint64_t)(L - 1) * npad};
    const cuuint64_t str[1] = {(cuuint64_t)HP * 2};
    const cuuint32_t box[2] = {128, 16};
    if (encode(reinterpret_cast<CUtensorMap*>(s->mact[p]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, s->act[p], dims, str,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled failed (activation blocks)";
      return cudaSuccess;
    }
  }
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p) {
      if (!enc(s->mb[b][p], s->xb[b][p], 3 * npad, 3 * LY_NBN)) {
        err = "cuTensorMapEncodeTiled failed";
        return cudaSuccess;
      }
      // one CTA's half of a pair tile's adjoint rows (120 of 240)
      if (!enc(s->mb2[b][p], s->xb[b][p], 3 * npad, 3 * LY_NBN / 2)) {
        err = "cuTensorMapEncodeTiled failed";
        return cudaSuccess;
      }
      // the backward GEMM's output boxes: 24 rows (8 nodes x 3) x 128 neurons
      const cuuint64_t dims[2] = {(cuuint64_t)HP, (cuuint64_t)3 * npad};
      const cuuint64_t str[1] = {(cuuint64_t)HP * 2};
      const cuuint32_t box[2] = {128, 24};
      if (encode(reinterpret_cast<CUtensorMap*>(s->mout[b][p]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, s->xb[b][p], dims,
                 str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (adjoint stores)";
        return cudaSuccess;
      }
    }
  // the stacked forward weights (W_1 .. W_L) and the reverse-mode stack
  // (transposes, W_0' hi / lo) in this path's 64 B swizzled tiles
  const long long rows_r = (long long)nh * HP + 128 + (long long)nh * HP + 256;
  if (!enc(s->wmap, tc.W, tc.rows_total, 128) || !enc(s->rmap, tc.WR, rows_r, 128)) {
    err = "cuTensorMapEncodeTiled failed";
    return cudaSuccess;
  }
  if (nh >= 1 && (!enc(s->mmap, s->mw, 6LL * HP, 128) || !enc(s->mdd[0], s->dd[0], npad, LY_NF) ||
                  !enc(s->mdd[1], s->dd[1], npad, LY_NF))) {
    err = "cuTensorMapEncodeTiled failed";
    return cudaSuccess;
  }
  if ((e = cudaFuncSetAttribute(lay_kernel<LY_BW0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ly_smem<LY_BW0>())) != cudaSuccess)
    return e;
  if (s->fp8 && nh >= 1) {
    // e4m3 codes of the hidden->hidden weights and their transposes
    std::vector<uint8_t> q((size_t)nh * HP * HP, 0), qt((size_t)nh * HP * HP, 0);
    for (int l = 1; l <= nh; ++l) {
      const int fi = net.widths[l], fo = net.widths[l + 1];
      std::vector<float> Wl((size_t)fo * fi);
      if ((e = cudaMemcpy(Wl.data(), net.W32 + net.w_off[l], Wl.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
      const float sc = net.fp8_scale[l];
      for (int i = 0; i < fo; ++i)
        for (int k = 0; k < fi; ++k) {
          const uint8_t c = (uint8_t)__nv_cvt_float_to_fp8(Wl[(size_t)i * fi + k] / sc, __NV_SATFINITE, __NV_E4M3);
          q[((size_t)(l - 1) * HP + i) * HP + k] = c;
          qt[((size_t)(l - 1) * HP + k) * HP + i] = c;
        }
    }
    if ((e = cudaMalloc(&s->q8, q.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(s->q8, q.data(), q.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&s->q8t, qt.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(s->q8t, qt.data(), qt.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    for (int p = 0; p < 3; ++p) {
      const size_t ab = (size_t)(L - 1) * npad * HP, bb = (size_t)3 * npad * HP;
      if ((e = cudaMalloc(&s->act8[p], ab)) != cudaSuccess) return e;
      if ((e = cudaMemset(s->act8[p], 0, ab)) != cudaSuccess) return e;
      for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&s->xb8[b][p], bb)) != cudaSuccess) return e;
        if ((e = cudaMemset(s->xb8[b][p], 0, bb)) != cudaSuccess) return e;
      }
    }
    // scales of the adjoints kept in e4m3 (D_l, l = 2 .. L-2): 448 / (8 x the
    // largest element of the adjoints of the linearised network (d = 1),
    // D_{L-1}[r] = W_{L-1}[r], D_l = W_l' D_{l+1}), so that typical
    // adjoints sit well inside e4m3's range with 8x headroom
    s->adj_scale.assign(L, 1.0f);
    {
      const int hl = net.widths[L - 1];
      std::vector<double> D((size_t)NO * hl);
      std::vector<float> WL((size_t)NO * hl);
      if ((e = cudaMemcpy(WL.data(), net.W32 + net.w_off[L - 1], WL.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
      for (size_t i = 0; i < D.size(); ++i) D[i] = WL[i];
      for (int l = L - 2; l >= 2; --l) {
        const int fi = net.widths[l], fo = net.widths[l + 1];
        std::vector<float> Wl((size_t)fo * fi);
        if ((e = cudaMemcpy(Wl.data(), net.W32 + net.w_off[l], Wl.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
          return e;
        std::vector<double> Dn((size_t)NO * fi, 0.0);
        double amax = 0.0;
        for (int r = 0; r < NO; ++r)
          for (int i = 0; i < fi; ++i) {
            double acc = 0.0;
            for (int k = 0; k < fo; ++k) acc += (double)Wl[(size_t)k * fi + i] * D[(size_t)r * fo + k];
            Dn[(size_t)r * fi + i] = acc;
            amax = std::max(amax, std::fabs(acc));
          }
        s->adj_scale[l] = amax > 0.0 ? (float)(448.0 / (8.0 * amax)) : 1.0f;
        D.swap(Dn);
      }
    }
    auto enc8 = [&](void* mp, void* ptr, long long rows, int box_rows) -> bool {
      const cuuint64_t dims[2] = {(cuuint64_t)HP, (cuuint64_t)rows};
      const cuuint64_t str[1] = {(cuuint64_t)HP};
      const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
      return encode(reinterpret_cast<CUtensorMap*>(mp), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, ptr, dims, str, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    bool ok = enc8(s->q8map, s->q8, (long long)nh * HP, 128) && enc8(s->q8tmap, s->q8t, (long long)nh * HP, 128);
    for (int p = 0; p < 3 && ok; ++p) {
      ok = enc8(s->a8map[p], s->act8[p], (long long)(L - 1) * npad, LY_NF) &&
           enc8(s->a8map2[p], s->act8[p], (long long)(L - 1) * npad, LY_NF / 2);
      for (int b = 0; b < 2 && ok; ++b)
        ok = enc8(s->b8map[b][p], s->xb8[b][p], 3 * npad, 3 * LY_NBN) &&
             enc8(s->b8map2[b][p], s->xb8[b][p], 3 * npad, 3 * LY_NBN / 2);
    }
    if (!ok) {
      err = "cuTensorMapEncodeTiled failed (FP8 operands)";
      return cudaSuccess;
    }
    if ((e = cudaFuncSetAttribute(lay_kernel<LY_FWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ly_smem<LY_FWD, true>())) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(lay_kernel<LY_BWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ly_smem<LY_BWD, true>())) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(lay2_kernel<LY_FWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Lb2<LY_FWD, true>::SMEM)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(lay2_kernel<LY_BWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Lb2<LY_BWD, true>::SMEM)) != cudaSuccess)
      return e;
  }
  if ((e = cudaFuncSetAttribute(lay_kernel<LY_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ly_smem<LY_FWD>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lay_kernel<LY_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ly_smem<LY_BWD>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lay2_kernel<LY_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Lb2<LY_BWD>::SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lay2_kernel<LY_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Lb2<LY_FWD>::SMEM)) != cudaSuccess)
    return e;

  return cudaFuncSetAttribute(lay_kernel<LY_JD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ly_smem<LY_JD>());
}

void mlp_lay_set_pair(rtn_ctx* ctx, bool pair) {
  if (ctx->net.tc.lay) ctx->net.tc.lay->pair_bwd = pair && (ctx->net.tc.h_pad / 128) % 2 == 0;
}

void mlp_lay_release(rtn_ctx* ctx) {
  LayState* s = ctx->net.tc.lay;
  if (!s) return;
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->side) cudaStreamDestroy(s->side);
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p)
      if (s->xb[b][p]) cudaFree(s->xb[b][p]);
  for (int p = 0; p < 2; ++p)
    if (s->act[p]) cudaFree(s->act[p]);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  if (s->mw) cudaFree(s->mw);
  if (s->w0s) cudaFree(s->w0s);
  for (int p = 0; p < 2; ++p)
    if (s->z[p]) cudaFree(s->z[p]);
  for (int p = 0; p < 2; ++p)
    if (s->dd[p]) cudaFree(s->dd[p]);
  if (s->q8) cudaFree(s->q8);
  if (s->q8t) cudaFree(s->q8t);
  for (int p = 0; p < 3; ++p) {
    if (s->act8[p]) cudaFree(s->act8[p]);
    for (int b = 0; b < 2; ++b)
      if (s->xb8[b][p]) cudaFree(s->xb8[b][p]);
  }
  delete s;
  ctx->net.tc.lay = nullptr;
}

cudaError_t mlp_lay_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  TcNet& tc = ctx->net.tc;
  LayState* s = tc.lay;
  if (!s) return cudaErrorInvalidValue;
  Net& net = ctx->net;
  const int L = net.n_layers, n = ctx->lay.n_nodes, HP = tc.h_pad, hs = s->hs;
  const int nh = L - 2;
  const size_t dstride = (size_t)s->npad * hs;
  cudaStream_t st = ctx->stream;
  const CUtensorMap* wmap = reinterpret_cast<const CUtensorMap*>(s->wmap);
  const CUtensorMap* rmap = reinterpret_cast<const CUtensorMap*>(s->rmap);
  auto maps = [&](unsigned char (&h)[128], unsigned char (&l)[128]) {
    LyMaps m;
    memcpy(&m.bh, h, sizeof(CUtensorMap));
    memcpy(&m.bl, l, sizeof(CUtensorMap));
    return m;
  };
  auto grid_of = [&](long long tiles) { return (int)std::min<long long>(tiles, std::max(1, tc.n_sm)); };
  const long long budget = tc.wait_cycles > 0 ? tc.wait_cycles : WAIT_CYCLES;
  const int stall = tc.inject_stall;
  const bool fp8 = s->fp8 && nh >= 1;
  const size_t dstride8 = (size_t)s->npad * hs;  // one layer of an FP8 piece array (bytes)
  auto maps8 = [&](unsigned char (&m)[3][128]) {
    LyMaps r;
    memcpy(&r.bh, m[0], sizeof(CUtensorMap));
    memcpy(&r.bl, m[1], sizeof(CUtensorMap));
    memcpy(&r.b3, m[2], sizeof(CUtensorMap));
    return r;
  };
  cudaError_t le = cudaSuccess;
  // an event before each launch when the pass is timed
  s->n_marks = 0;
  auto mark = [&](int kind) {
    if (!s->timing || s->n_marks >= (int)s->ev.size()) return;
    cudaEventRecord(s->ev[s->n_marks], st);
    s->kind[s->n_marks++] = kind;
  };
  // input layer -> values buffer 0, d_1: z split into BF16 hi + lo, then a
  // GEMM against W_0 hi / lo with the forward epilogue
  const int gf = (n + LY_NF - 1) / LY_NF;
  {
    const long long ne = (long long)n * NZ;
    mark(0);
    lay_z_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(x, u, ctx->lay.node_inst, n, s->z[0], s->z[1]);
    LyArgs a{};
    a.a_row0 = 0;
    a.a_lo = HP;
    a.m_rows = net.widths[1];
    a.mts = (net.widths[1] + 127) / 128;
    a.nkb = 1;
    a.n_nodes = n;
    a.n_groups = gf;
    a.hs = hs;
    a.bias = tc.b0;
    a.yh = s->act[0];
    a.yl = s->act[1];
    if (fp8) {
      a.y8h = s->act8[0];
      a.y8m = s->act8[1];
      a.y8l = s->act8[2];
    }
    a.err = tc.err;
    a.wait_cycles = budget;
    a.stall = stall;
    mark(1);
    lay_kernel<LY_IN><<<grid_of((long long)gf * a.mts), Ly<LY_IN>::THREADS, ly_smem<LY_IN>(), st>>>(
        *reinterpret_cast<const CUtensorMap*>(s->mw0), maps(s->mz[0], s->mz[1]), a);
  }
  // forward hidden layers: GEMM g reads a_{g+1}, writes a_{g+2}
  for (int g = 0; g < nh; ++g) {
    const int ho = net.widths[g + 2];
    LyArgs a{};
    a.a_row0 = g * HP;
    a.m_rows = ho;
    a.mts = (ho + 127) / 128;
    a.nkb = HP / LY_KB;
    a.n_nodes = n;
    a.n_groups = gf;
    a.hs = hs;
    a.bias = tc.bias + (size_t)g * HP;
    a.b_row0 = g * s->npad;
    if (g == nh - 1) {  // d_{L-1}: the B operand of the folded first backward GEMM
      a.dh = s->dd[0];
      a.dl = s->dd[1];
    }
    a.yh = s->act[0] + (size_t)(g + 1) * dstride;
    a.yl = s->act[1] + (size_t)(g + 1) * dstride;
    a.err = tc.err;
    a.wait_cycles = budget;
    a.stall = stall;
    mark(2);
    if (fp8) {
      // e4m3 W_{g+1} against the pieces of 448 a_{g+1}; a_{g+2} out as pieces,
      // and as BF16 hi + lo where a BF16 GEMM reads it (a_{L-2}, a_{L-1})
      a.nkb = HP / 64;
      a.sc = net.fp8_scale[g + 1] / 448.0f;
      a.y8h = s->act8[0] + (size_t)(g + 1) * dstride8;
      a.y8m = s->act8[1] + (size_t)(g + 1) * dstride8;
      a.y8l = s->act8[2] + (size_t)(g + 1) * dstride8;
      if (g < nh - 2) a.yh = a.yl = nullptr;
      if (s->pair_bwd && a.mts % 2 == 0) {
        // pair tiles of 256 neurons: each CTA loads half of the pieces' node rows
        const long long pt = (long long)gf * (a.mts / 2);
        const int pairs = (int)std::min<long long>(pt, std::max(1, tc.n_sm / 2));
        lay2_kernel<LY_FWD, true><<<2 * pairs, Lb2<LY_FWD, true>::THREADS, Lb2<LY_FWD, true>::SMEM, st>>>(
            *reinterpret_cast<const CUtensorMap*>(s->q8map), maps8(s->a8map2), a);
      } else {
        lay_kernel<LY_FWD, true><<<grid_of((long long)gf * a.mts), Ly<LY_FWD, true>::THREADS,
                                   ly_smem<LY_FWD, true>(), st>>>(*reinterpret_cast<const CUtensorMap*>(s->q8map),
                                                                  maps8(s->a8map), a);
      }
    } else {
      LyMaps m = maps(s->ma[0], s->ma[1]);
      memcpy(&m.oh, s->mact[0], sizeof(CUtensorMap));  // a_{g+2}: box 128 neurons x 16 nodes
      memcpy(&m.ol, s->mact[1], sizeof(CUtensorMap));
      a.out_row0 = (g + 1) * s->npad;
      if (s->pair_bwd && a.mts % 2 == 0) {
        // pair tiles of 256 neurons: each CTA loads half of the tile's 256 node rows
        memcpy(&m.bh, s->ma2[0], sizeof(CUtensorMap));
        memcpy(&m.bl, s->ma2[1], sizeof(CUtensorMap));
        const long long pt = (long long)gf * (a.mts / 2);
        const int pairs = (int)std::min<long long>(pt, std::max(1, tc.n_sm / 2));
        lay2_kernel<LY_FWD><<<2 * pairs, Lb2<LY_FWD>::THREADS, Lb2<LY_FWD>::SMEM, st>>>(*wmap, m, a);
      } else {
        lay_kernel<LY_FWD><<<grid_of((long long)gf * a.mts), Ly<LY_FWD>::THREADS, ly_smem<LY_FWD>(), st>>>(*wmap, m,
                                                                                                             a);
      }
    }
  }
  // f_D (and, with no hidden->hidden layer, the last layer's adjoints into
  // adjoint buffer 0).  With hidden->hidden layers f_D reads only a_{L-1}
  // and nothing in the pass reads f_D, so it runs on the side stream beside
  // the first backward GEMM (launched first, so that its CTAs are placed
  // before the output layer's blocks take the SMs' other slots) and joins at
  // the pass's end; in a timed pass it stays in line
  const bool side_fd = nh >= 1 && net.widths[L - 1] % 8 == 0 && !s->timing;
  if (side_fd && (le = cudaEventRecord(s->ev_fork, st)) != cudaSuccess) return le;
  {
    const __nv_bfloat16* aLh = s->act[0] + (size_t)(L - 2) * dstride;
    const __nv_bfloat16* aLl = s->act[1] + (size_t)(L - 2) * dstride;
    const long long warps = n;
    const int blocks = (int)std::min<long long>((warps + 7) / 8, 148LL * 64);
    mark(3);
    if (side_fd) {
      // launched on the side stream after the first backward GEMM (below)
    } else if (nh >= 1 && net.widths[L - 1] % 8 == 0)
      lay_fd_kernel<<<blocks, 256, 0, st>>>(tc.WL32, tc.bias + (size_t)nh * HP, net.widths[L - 1], n, hs, aLh, aLl,
                                            fD, HP);
    else
      lay_out_kernel<<<blocks, 256, 0, st>>>(tc.WL32, tc.bias + (size_t)nh * HP, net.widths[L - 1], n, hs, aLh, aLl,
                                             fD, nh >= 1 ? nullptr : s->xb[0][0], s->xb[0][1], HP);
  }
  // first backward layer with the last layer's adjoints folded in:
  // D_{L-2}[n, r] = d_{L-2} (.) (M_r d_{L-1}[n]) -> adjoint buffer 0
  if (nh >= 1) {
    LyArgs a{};
    a.a_row0 = 0;
    a.a_lo = 3 * HP;
    a.m_rows = net.widths[L - 2];
    a.mtpr = HP / 128;
    a.mts = 3 * a.mtpr;
    a.nkb = HP / LY_KB;
    a.n_nodes = n;
    a.n_groups = gf;
    a.hs = hs;
    a.ah = s->act[0] + (size_t)(L - 3) * dstride;
    a.al = s->act[1] + (size_t)(L - 3) * dstride;
    a.yh = s->xb[0][0];
    a.yl = s->xb[0][1];
    if (fp8 && nh >= 2) {  // D_{L-2} feeds an FP8 backward GEMM: e4m3 pieces
      a.yh = a.yl = nullptr;
      a.y8h = s->xb8[0][0];
      a.y8m = s->xb8[0][1];
      a.y8l = s->xb8[0][2];
      a.s8 = s->adj_scale[L - 2];
    }
    a.err = tc.err;
    a.wait_cycles = budget;
    a.stall = stall;
    LyMaps m;
    memcpy(&m.bh, s->mdd[0], sizeof(CUtensorMap));
    memcpy(&m.bl, s->mdd[1], sizeof(CUtensorMap));
    memcpy(&m.sh, s->mact[0], sizeof(CUtensorMap));
    memcpy(&m.sl, s->mact[1], sizeof(CUtensorMap));
    a.act_row0 = (L - 3) * s->npad;
    mark(4);
    lay_kernel<LY_BW0><<<grid_of((long long)gf * a.mts), Ly<LY_BW0>::THREADS, ly_smem<LY_BW0>(), st>>>(
        *reinterpret_cast<const CUtensorMap*>(s->mmap), m, a);
  }
  if (side_fd) {
    const long long warps = n;
    const int blocks = (int)std::min<long long>((warps + 7) / 8, 148LL * 64);
    if ((le = cudaStreamWaitEvent(s->side, s->ev_fork, 0)) != cudaSuccess) return le;
    lay_fd_kernel<<<blocks, 256, 0, s->side>>>(tc.WL32, tc.bias + (size_t)nh * HP, net.widths[L - 1], n, hs,
                                               s->act[0] + (size_t)(L - 2) * dstride,
                                               s->act[1] + (size_t)(L - 2) * dstride, fD, HP);
    if ((le = cudaGetLastError()) != cudaSuccess || (le = cudaEventRecord(s->ev_join, s->side)) != cudaSuccess)
      return le;
  }
  // the other backward hidden layers: D_l = d_l (.) (W_l' D_{l+1}), l = L - 3 .. 1
  const int gb = (n + LY_NBN - 1) / LY_NBN;
  const int tb = nh * HP + 128;  // first transposed row in the reverse-mode stack
  for (int k = 1; k < nh; ++k) {
    const int l = L - 2 - k, src = (k - 1) & 1, dst = src ^ 1, hl = net.widths[l];
    LyArgs a{};
    a.a_row0 = tb + (l - 1) * HP;
    a.m_rows = hl;
    a.mts = (hl + 127) / 128;
    a.nkb = HP / LY_KB;
    a.n_nodes = n;
    a.n_groups = gb;
    a.hs = hs;
    a.ah = s->act[0] + (size_t)(l - 1) * dstride;
    a.al = s->act[1] + (size_t)(l - 1) * dstride;
    a.yh = s->xb[dst][0];
    a.yl = s->xb[dst][1];
    a.err = tc.err;
    a.wait_cycles = budget;
    a.stall = stall;
    mark(5);
    if (fp8) {
      // e4m3 W_l' against the pieces of D_{l+1} * s_{l+1}; d_l from the pieces
      // of 448 a_l; D_l out as pieces (scale s_l) or, for the Jacobian GEMM
      // (l = 1), as BF16 hi + lo
      a.nkb = HP / 64;
      a.sc = net.fp8_scale[l] / s->adj_scale[l + 1];
      a.a8h = s->act8[0] + (size_t)(l - 1) * dstride8;
      a.a8m = s->act8[1] + (size_t)(l - 1) * dstride8;
      a.a8l = s->act8[2] + (size_t)(l - 1) * dstride8;
      if (l >= 2) {
        a.yh = a.yl = nullptr;
        a.y8h = s->xb8[dst][0];
        a.y8m = s->xb8[dst][1];
        a.y8l = s->xb8[dst][2];
        a.s8 = s->adj_scale[l];
      }
      a.a_row0 = (l - 1) * HP;
      if (s->pair_bwd && a.mts % 2 == 0) {
        // pair tiles of 256 neurons: each CTA loads half of the pieces' adjoint rows
        const long long pt = (long long)gb * (a.mts / 2);
        const int pairs = (int)std::min<long long>(pt, std::max(1, tc.n_sm / 2));
        lay2_kernel<LY_BWD, true><<<2 * pairs, Lb2<LY_BWD, true>::THREADS, Lb2<LY_BWD, true>::SMEM, st>>>(
            *reinterpret_cast<const CUtensorMap*>(s->q8tmap), maps8(s->b8map2[src]), a);
      } else {
        lay_kernel<LY_BWD, true><<<grid_of((long long)gb * a.mts), LY_THREADS, ly_smem<LY_BWD, true>(), st>>>(
            *reinterpret_cast<const CUtensorMap*>(s->q8tmap), maps8(s->b8map[src]), a);
      }
    } else {
      LyMaps m = maps(s->mb[src][0], s->mb[src][1]);
      memcpy(&m.sh, s->mact[0], sizeof(CUtensorMap));
      memcpy(&m.sl, s->mact[1], sizeof(CUtensorMap));
      memcpy(&m.oh, s->mout[dst][0], sizeof(CUtensorMap));
      memcpy(&m.ol, s->mout[dst][1], sizeof(CUtensorMap));
      a.act_row0 = (l - 1) * s->npad;
      if (s->pair_bwd && a.mts % 2 == 0) {
        // pair tiles of 256 neurons: each CTA loads half of the adjoint rows
        memcpy(&m.bh, s->mb2[src][0], sizeof(CUtensorMap));
        memcpy(&m.bl, s->mb2[src][1], sizeof(CUtensorMap));
        const long long pt = (long long)gb * (a.mts / 2);
        const int pairs = (int)std::min<long long>(pt, std::max(1, tc.n_sm / 2));
        lay2_kernel<LY_BWD><<<2 * pairs, Lb2<LY_BWD>::THREADS, Lb2<LY_BWD>::SMEM, st>>>(*rmap, m, a);
      } else {
        lay_kernel<LY_BWD><<<grid_of((long long)gb * a.mts), Ly<LY_BWD>::THREADS, ly_smem<LY_BWD>(), st>>>(*rmap, m,
                                                                                                           a);
      }
    }
  }
  // J_D = W_0' D_1 (W_0' hi and lo rows)
  {
    const int src = nh >= 1 ? (nh - 1) & 1 : 0;
    LyArgs a{};
    a.a_row0 = tb + nh * HP;
    a.a_lo = 128;
    a.m_rows = NZ;
    a.mts = 1;
    a.nkb = HP / LY_KB;
    a.n_nodes = n;
    a.n_groups = gb;
    a.hs = hs;
    a.JD = JD;
    a.err = tc.err;
    a.wait_cycles = budget;
    a.stall = stall;
    mark(6);
    lay_kernel<LY_JD><<<grid_of(gb), LY_THREADS, ly_smem<LY_JD>(), st>>>(*rmap, maps(s->mb[src][0], s->mb[src][1]),
                                                                          a);
  }
  if (s->timing && s->n_marks < (int)s->ev.size()) cudaEventRecord(s->ev[s->n_marks], st);
  if (side_fd && (le = cudaStreamWaitEvent(st, s->ev_join, 0)) != cudaSuccess) return le;
  return cudaGetLastError();
}

cudaError_t mlp_lay_timing(rtn_ctx* ctx, bool enable) {
  LayState* s = ctx->net.tc.lay;
  if (!s) return cudaErrorInvalidValue;
  if (enable && s->ev.empty()) {
    const int n_ev = 2 * ctx->net.n_layers + 2;  // 2 L launches and the end
    s->ev.resize(n_ev);
    s->kind.assign(n_ev, -1);
    for (auto& e : s->ev) {
      const cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
    }
  }
  s->timing = enable;
  s->n_marks = 0;
  return cudaSuccess;
}

cudaError_t mlp_lay_times(rtn_ctx* ctx, float* ms, int* kind, int cap, int* count) {
  LayState* s = ctx->net.tc.lay;
  if (!s || s->ev.empty()) return cudaErrorInvalidValue;
  const int n = s->n_marks;
  cudaError_t e = cudaEventSynchronize(s->ev[n]);
  for (int i = 0; i < n && i < cap && e == cudaSuccess; ++i) {
    e = cudaEventElapsedTime(ms + i, s->ev[i], s->ev[i + 1]);
    kind[i] = s->kind[i];
  }
  *count = n;
  return e;
}

}  // namespace rtn

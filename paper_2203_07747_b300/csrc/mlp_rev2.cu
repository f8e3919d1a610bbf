// mlp_rev2.cu -- (a1, reverse mode) residual network value f_D and input
// Jacobian J_D on CTA pairs: the computation of mlp_rev.cu (one value column
// forward, three output adjoints backward per node, Sec. III-A Eq. 4) with
// tcgen05.mma cta_group::2, M = 256 weight rows per instruction.
//
// Why pairs: an M = 128 MMA reads its 128 x 16 weight slice (4 KB) from
// shared memory, and the TMA that filled the slice wrote the same 4 KB; with
// one CTA an MMA of N <= 128 columns is bound by those shared-memory bytes,
// not by the tensor pipe.  On a pair each CTA supplies its own 128 weight
// rows and half of the N activation columns, so an N = 256 MMA moves 12 KB
// through each SM's shared memory in the 128 cycles it computes.
//
// Tile: NPC = 42 nodes per pair.  Rank 0 holds the hi, rank 1 the lo BF16
// part of every activation column (same offsets in both CTAs):
//   forward:  C_F = 64 value columns per CTA (42 used), N = 128;
//   backward: C_B = 128 adjoint columns per CTA (3n + i, 126 used), N = 256.
// The activation buffer X is N-major with 64 columns in the forward pass and
// 128 in the backward pass.  The forward layout fills half of X, so forward
// GEMMs alternate between the two halves: GEMM g (g <= nh) reads half g % 2
// and its epilogue writes the other, whose last reader (GEMM g - 1) has
// completed once GEMM g's accumulator has; the backward layout covers all of
// X (the passes meet only after the MMAs have read every block).  GEMMs of a tile, all on the
// stacked weights of the single-CTA reverse kernel:
//   g < nh        W_{g+1}  forward hidden layer (a_{g+2} = tanh(W a + b))
//   g = nh        W_L      output layer (rank 0's rows only): f_D
//   nh < g <= 2nh W_l'     backward hidden layer, l = 2 nh + 1 - g
//   g = 2 nh + 1  W_0'     J_D = W_0' D_1, hi rows then lo rows (rank 0 only)
// with d_l = 1 - a_l^2 in a per-pair FP32 scratch (node-major, L2-resident):
// D_L = d_L (.) W_L' (SIMT), D_l = d_l (.) (W_l' D_{l+1}).
//
// Exchange of a block (128 rows of X) between the CTAs: block j is produced
// by rank j % 2 (the accumulator rows it holds); the producer writes its own half into its X, stages the peer's half
// and pushes it with a bulk copy that completes on a barrier of the peer; the
// exchange warps relay the completion and free the staging block.  The input
// layer (FP32 dot products over the 17 inputs) is exchanged the same way:
// each CTA computes the rows of its own blocks for every node.  The
// last-layer adjoints (one product per value) are not exchanged: each CTA
// computes its own half for every row, after a cluster-scope barrier has made
// the peer's d_L visible; all 16 epilogue warps publish on rank 0's xin[j].
// The notice that the MMAs have read block j (xfree) reaches both CTAs once
// per GEMM; every wait on it names its completion by the GEMM count.
// Every wait is bounded (RTN_E_TIMEOUT in the device flag).
#include <algorithm>

#include "tc_pair.cuh"

namespace rtn {
namespace {

constexpr int R2_NPC = 42;        // nodes per pair tile
constexpr int R2_CF = 64;         // forward columns per CTA
constexpr int R2_CB = 128;        // backward columns per CTA
constexpr int R2_THREADS = THREADS + 32;  // warp 10: exchange
constexpr uint32_t R2_SBYTES = 128u * R2_CB * 2u;  // staging block (backward size)

struct Rev2Args {
  const float* x;
  const float* u;
  const int* node_inst;
  int n_nodes;
  const float* W0;    // [17][HP] FP32 input layer (transposed)
  const float* b0;    // [HP]
  const float* bias;  // hidden biases [n_hidden_mm * HP] then output [>= 3]
  const float* WL;    // [3][HP] FP32 output layer
  int HP;
  int n_hidden_mm;
  uint32_t tmem_cols;
  float* fD;
  float* JD;
  float* dscr;  // [pairs][n_hidden_mm + 1][R2_NPC][HP] FP32: d_l of the tile
  int* err;
  unsigned long long* trace;
};

// GEMM g of a tile: weight row base, M tiles of 256 rows, kind
struct Rev2Layer {
  int row0;     // first weight row of M tile 0 (rank r adds 128 r)
  int mts;      // M tiles (1 for the single-tile GEMMs)
  bool bwd;     // backward: N = 256, else N = 128
  bool single;  // rank 0's 128 rows only (output layer, W_0')
  bool two;     // W_0': a second K pass over the lo rows (+128)
};

__device__ __forceinline__ Rev2Layer rev2_layer(int g, int nh, int HP) {
  const int n_mt2 = HP / 256, tb = nh * HP + 128;
  if (g < nh) return {g * HP, n_mt2, false, false, false};
  if (g == nh) return {nh * HP, 1, false, true, false};
  if (g < 2 * nh + 1) return {tb + (2 * nh - g) * HP, n_mt2, true, false, false};
  return {tb + nh * HP, 1, true, true, true};
}

// phase trace of CTA 0 (rank 0): same entries as the single-CTA reverse kernel
__device__ __forceinline__ void rev2_trace(const Rev2Args& a, int it, int g, int n_gemm, int f,
                                           unsigned long long v) {
  const int idx = (it * (n_gemm + 1) + g) * 8 + f;
  if (idx < (1 << 16)) a.trace[idx] = v;
}

// byte offset of (row k, column c) in an N-major X of cx columns
__device__ __forceinline__ uint32_t xoff_n(int cx, int k, int c) {
  return (uint32_t)(k >> 3) * (uint32_t)(cx * 16) + (uint32_t)(c >> 3) * 128u + (uint32_t)(k & 7) * 16u +
         (uint32_t)(c & 7) * 2u;
}

// hi and lo BF16 parts of v packed in pairs: h = bf16(v), l = bf16(v - h)
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& h, uint32_t& l) {
  h = pack_bf16(v0, v1);
  l = pack_res(v0, v1, h);
}

template <int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(R2_THREADS, 1)
    mlp_rev2_kernel(const __grid_constant__ CUtensorMap tmap, Rev2Args a) {
  constexpr int NPC = R2_NPC, NZV = NPC * NZ;
  constexpr int MT = 2, NB = 4;  // accumulator slots, 128-row blocks (hidden width <= 512)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t rank = cluster_rank();
  const int HP = a.HP, n_mt2 = HP / 256, nkb = HP / 64, nblk = HP / 128;
  const int nh = a.n_hidden_mm, n_gemm = 2 * nh + 2;
  const int n_tiles = (a.n_nodes + NPC - 1) / NPC;
  const int pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t sbase = sraw + pad;
  const uint32_t xbytes = (uint32_t)R2_CB * HP * 2u;
  uint8_t* X = sm;              // X_hi (rank 0) / X_lo (rank 1)
  uint8_t* S = sm + xbytes;     // staging block for the peer's half
  const uint32_t x_s = sbase, s_s = sbase + xbytes;
  const uint32_t x_rem = mapa(x_s, rank ^ 1u);  // the peer's X
  const bool lo_local = rank == 1;
  const uint32_t w_s = sbase + xbytes + R2_SBYTES;
  uint8_t* tail_area = sm + xbytes + R2_SBYTES + STAGES * WT_BYTES;
  const uint32_t bar_s = smem_u32(tail_area);
  auto full_bar = [&](int s) { return bar_s + 8u * s; };
  auto empty_bar = [&](int s) { return bar_s + 8u * (STAGES + s); };
  auto acc_full = [&](int m) { return bar_s + 8u * (2 * STAGES + m); };
  auto tmem_free = [&](int m) { return bar_s + 8u * (2 * STAGES + MT + m); };
  auto xready = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + j); };
  auto xfree = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + NB + j); };
  auto lo_in = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + 2 * NB + j); };
  auto xin = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + 3 * NB + j); };
  const uint32_t s_full = bar_s + 8u * (2 * STAGES + 2 * MT + 4 * NB);
  const uint32_t s_free = s_full + 8u, z_full = s_full + 16u, z_free = s_full + 24u;
  const uint32_t d_ready = s_full + 32u, bwd_done = s_full + 40u;
  constexpr int NBAR = 2 * STAGES + 2 * MT + 4 * NB + 6;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail_area + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* zbuf = reinterpret_cast<float*>(tail_area + 8 * NBAR + 16);
  float* dscr = a.dscr + (size_t)pair * (nh + 1) * NPC * HP;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int m = 0; m < MT; ++m) {
      mbar_init(acc_full(m), 1);
      mbar_init(tmem_free(m), 2 * EPI_WARPS);
    }
    for (int j = 0; j < NB; ++j) {
      // even blocks: rank 0's own half + the relay of its lo half; odd blocks:
      // one arrival of rank 1 plus the bytes of its hi half
      mbar_init(xready(j), (j & 1) ? 1 : 2);
      mbar_init(xfree(j), 1);
      mbar_init(lo_in(j), 1);
      mbar_init(xin(j), 2 * EPI_WARPS);
    }
    mbar_init(s_full, EPI_WARPS);
    mbar_init(s_free, 1);
    mbar_init(z_full, EPI_WARPS);
    mbar_init(z_free, EPI_WARPS);
    mbar_init(bwd_done, EPI_WARPS);
    mbar_init(d_ready, 2 * EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero this CTA's X (padding columns stay 0) and S before the peer may copy into X
  for (uint32_t o = threadIdx.x * 16u; o < xbytes + R2_SBYTES; o += R2_THREADS * 16u)
    *reinterpret_cast<uint4*>(sm + o) = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
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
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(mapa(smem_u32(tmem_slot), 0))
                 : "memory");
    if (other != tmem) {
      atomicExch(a.err, (int)RTN_E_UNSUPPORTED);
      *abort_flag = 1;
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(mapa(smem_u32((const void*)abort_flag), 0)),
                   "r"(1)
                   : "memory");
    }
  }
  cluster_sync();
  const bool run = (*abort_flag == 0);

  if (run && warp == 0) {
    // ---------------- TMA producer (both CTAs; whole warp, one elected lane
    // issues): this CTA's 128 rows of each 256-row tile, K blocks in the
    // order the MMAs use them (1, 0, 3, 2, ...)
    if (lane == 0)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    {
      const uint32_t full0 = mapa(full_bar(0), 0);  // stage barriers of rank 0
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs)
        for (int g = 0; g < n_gemm && ok; ++g) {
          const Rev2Layer L = rev2_layer(g, nh, HP);
          const int nks = L.two ? 2 * nkb : nkb;
          for (int m = 0; m < L.mts && ok; ++m)
            for (int kb = 0; kb < nks && ok; ++kb) {
              if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err))) break;
              if (elect_one()) {
                // single-tile GEMMs: rank 1's half is padding whose products
                // land in accumulator rows nobody reads: not loaded
                const bool load = !L.single || rank == 0;
                if (rank == 0) mbar_expect_tx(full_bar(s), (L.single ? 1 : 2) * WT_BYTES);
                const int kk = (kb % nkb) ^ 2;
                if (load)
                  tma_load_2d_pair(w_s + s * WT_BYTES, &tmap, kk * 64,
                                   L.row0 + m * 256 + (int)rank * 128 + (kb >= nkb ? 128 : 0), full0 + 8u * s);
              }
              __syncwarp();
              if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
        }
      // tail: every stage released, so no commit from the peer lands after exit
      for (int i = 0; i < STAGES && ok; ++i) {
        ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err);
        if (++s == STAGES) { s = 0; ph ^= 1u; }
      }
    }
  } else if (run && warp == 1) {
    if (rank == 0) {
      // ---------------- MMA issuer of the pair (whole warp, one elected lane issues)
      constexpr uint32_t id_f = idesc_bf16(256, 2 * R2_CF) | (1u << 16);  // B is N-major
      constexpr uint32_t id_b = idesc_bf16(256, 2 * R2_CB) | (1u << 16);
      int s = 0;
      uint32_t ph = 0, used = 0, tf_par = 0, xr_par = 0, xi_par = 0;
      bool ok = true;
      const bool tr = RTN_TRACE && a.trace != nullptr && blockIdx.x == 0;
      WaitClock wc(tr);
      for (int tile = pair, it = 0; tile < n_tiles && ok; tile += n_pairs, ++it)
        for (int g = 0; g < n_gemm && ok; ++g) {
          const Rev2Layer L = rev2_layer(g, nh, HP);
          const int nks = L.two ? 2 * nkb : nkb;
          const uint32_t idesc = L.bwd ? id_b : id_f;
          const uint32_t lbo = (L.bwd ? R2_CB : R2_CF) * 16u;
          const uint32_t xs_g = x_s + (L.bwd ? 0u : (uint32_t)(g & 1) * (xbytes / 2u));  // forward half
          long long w_x = 0, w_w = 0, w_t = 0;
          if (tr && lane == 0) rev2_trace(a, it, g, n_gemm, 0, gtime());
          for (int m = 0; m < L.mts && ok; ++m) {
            // single-tile GEMMs use slot 1 so that the next GEMM's first M
            // tile need not wait for their read-out
            const int slot = L.single ? 1 : m;
            if (used & (1u << slot)) {
              wc.start();
              ok = mbar_wait_cl_warp(tmem_free(slot), (tf_par >> slot) & 1u, abort_flag, a.err);
              wc.stop(w_t);
              if (!ok) break;
              tf_par ^= 1u << slot;
            }
            used |= 1u << slot;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(slot * 256);
            for (int kb = 0; kb < nks && ok; ++kb) {
              const int kk = (kb % nkb) ^ 2, j = kk >> 1;
              if (m == 0 && kb < nkb && (kb & 1) == 0) {
                wc.start();
                if (g == nh + 1) {  // the last-layer adjoints (both CTAs publish on xin)
                  ok = mbar_wait_cl_warp(xin(j), (xi_par >> j) & 1u, abort_flag, a.err);
                  xi_par ^= 1u << j;
                } else {
                  ok = mbar_wait_cl_warp(xready(j), (xr_par >> j) & 1u, abort_flag, a.err);
                  xr_par ^= 1u << j;
                }
                wc.stop(w_x);
                if (!ok) break;
                tc_fence_after();
              }
              wc.start();
              ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err);
              wc.stop(w_w);
              if (!ok) break;
              tc_fence_after();
              const uint32_t as = w_s + s * WT_BYTES;
              uint64_t ad[4], bd[4];
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t bo = (uint32_t)(kk * 4 + ks) * 2u * lbo;  // 16 k = 2 k-groups
                ad[ks] = wdesc(as, ks);
                bd[ks] = xdesc(xs_g + bo, lbo);
              }
              mma2_bf16_x4(d, ad, bd, idesc, kb != 0);
              commit2(empty_bar(s), 3);
              if (++s == STAGES) { s = 0; ph ^= 1u; }
              // the GEMM's last read of block j: its producer may rewrite it
              if (m == L.mts - 1 && kb >= nks - nkb && (kb & 1)) commit2(xfree(j), 3);
            }
            if (ok) commit2(acc_full(slot), 3);
          }
          if (tr && lane == 0) {
            rev2_trace(a, it, g, n_gemm, 1, gtime());
            rev2_trace(a, it, g, n_gemm, 4, w_x);
            rev2_trace(a, it, g, n_gemm, 5, w_w);
            rev2_trace(a, it, g, n_gemm, 6, w_t);
          }
        }
    }
  } else if (run && warp == THREADS / 32) {
    if (lane == 0) {
      // ---------------- exchange warp: the exchanged blocks of every tile
      // (the input layer, nh forward layers, nh backward layers), in the
      // order their producers publish them
      const uint32_t xr0 = mapa(xready(0), 0);
      const uint32_t sfree_peer = mapa(s_free, rank ^ 1u);
      uint32_t par = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs)
        for (int l = 0; l < 2 * nh + 1 && ok; ++l)
          for (int m = 0; m < n_mt2 && ok; ++m) {
            if (rank == 1) {
              // rank 0's lo half of block 2m has landed here
              const int j = 2 * m;
              if (!(ok = mbar_wait_cl(lo_in(j), (par >> j) & 1u, abort_flag, a.err))) break;
              par ^= 1u << j;
              arrive_cluster(xr0 + 8u * j);
            } else {
              // rank 1's hi half of block 2m + 1 has landed here
              const int j = 2 * m + 1;
              if (!(ok = mbar_wait_cl(xready(j), (par >> j) & 1u, abort_flag, a.err))) break;
              par ^= 1u << j;
            }
            arrive_cluster(sfree_peer);  // the copy has read the peer's staging block
          }
    }
  } else if (run && warp >= 2) {
    // ---------------- epilogue warps (both CTAs)
    const int e = warp - 2;           // 0..7
    const int q = warp & 3;           // TMEM lane quadrant
    const int half = e >> 2;          // forward: nodes 24 half ..; backward: columns 64 half ..
    const int et = threadIdx.x - 64;  // 0..255
    const bool elected = (e == 0 && lane == 0);  // publishes each block
    auto ldz = [&](int node, int jj) -> float {
      if (node >= a.n_nodes) return 0.0f;
      return jj < NX ? a.x[(size_t)(node + a.node_inst[node]) * NX + jj]
                     : a.u[(size_t)node * NU + (jj - NX)];
    };
    // the tile's inputs z (NPC x 17 values, up to three per epilogue thread)
    static_assert(NZV <= 768, "z staging");
    float zpref[3];
    auto prefetch_z = [&](int tile) {
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        const int e2 = et + 256 * h;
        zpref[h] = e2 < NZV ? ldz(tile * NPC + e2 / NZ, e2 % NZ) : 0.0f;
      }
    };
    if (pair < n_tiles) prefetch_z(pair);
    uint32_t acc_par = 0, sf_ph = 0, ss_par = 0, zf_par = 0, zr_ph = 0, dr_par = 0, bd_par = 0;
    bool ok = true;
    const uint32_t tf0 = mapa(tmem_free(0), 0);
    const uint32_t xr0 = mapa(xready(0), 0), lo1 = mapa(lo_in(0), 1), xi0 = mapa(xin(0), 0);
    const uint32_t dr0 = mapa(d_ready, 0), dr1 = mapa(d_ready, 1);
    // xfree[j] completes once per GEMM: completion c (from 1) of the pair's
    // tile it, GEMM g is c = n_gemm it + g + 1; wait parity (c - 1) & 1
    auto xfree_par = [&](int it_, int g) -> uint32_t { return (uint32_t)(n_gemm * it_ + g) & 1u; };
    const bool etr = RTN_TRACE && a.trace != nullptr && blockIdx.x == 0 && e == 0 && lane == 0;
    long long ew = 0;
    auto wwait = [&](uint32_t bar, uint32_t par) -> bool {
      int w_ok = 0;
      if (lane == 0) {
        const long long t0 = etr ? clock64() : 0;
        w_ok = mbar_wait(bar, par, abort_flag, a.err);
        if (etr) ew += clock64() - t0;
      }
      return __shfl_sync(0xffffffffu, w_ok, 0) != 0;
    };
    auto mark = [&](int it_, int g, int f) {
      if (etr) rev2_trace(a, it_, g, n_gemm, f, gtime());
    };
    // step stamps of one M tile's epilogue (traced thread): entry 32768 +
    // ((it * n_gemm + g) * 2 + m) * 8 + f
    auto stamp = [&](int it_, int g, int m, int f) {
      if (etr) {
        const int idx = 32768 + ((it_ * n_gemm + g) * 2 + m) * 8 + f;
        if (idx < (1 << 16)) a.trace[idx] = gtime();
      }
    };
    auto mark_end = [&](int it_, int g) {
      if (etr) {
        rev2_trace(a, it_, g, n_gemm, 3, gtime());
        rev2_trace(a, it_, g, n_gemm, 7, ew);
      }
      ew = 0;
    };
    // d_l of row r: node n at dptr(l, r)[n * HP]
    auto dptr = [&](int layer, int r) -> float* { return dscr + (size_t)layer * NPC * HP + r; };
    // before the staging block is rewritten: the previous copy has landed
    auto wait_staging = [&]() -> bool {
      if (!wwait(s_free, sf_ph ^ 1u)) return false;
      sf_ph ^= 1u;
      return true;
    };
    // after every warp wrote its rows of block j: publish the own half, push
    // the peer's half (`bytes` = one block of the current layout)
    auto block_end = [&](int j, uint32_t bytes, uint32_t base) -> bool {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(s_full);
      int p_ok = 1;
      if (elected) {
        p_ok = mbar_wait(s_full, ss_par, abort_flag, a.err);
        ss_par ^= 1u;
        if (p_ok) {
          const uint32_t bar = (rank == 0 ? lo1 : xr0) + 8u * j;
#pragma unroll
          for (int c = 0; c < 4; ++c)  // four copies in flight, issued first
            bulk_copy_to_peer(x_rem + base + (uint32_t)j * bytes + c * (bytes / 4), s_s + c * (bytes / 4),
                              bytes / 4, bar);
          if (rank == 0) {
            mbar_arrive(xready(j));                        // own hi half
            arrive_expect_tx_cluster_relaxed(bar, bytes);  // the copy's bytes
          } else {
            arrive_expect_tx_cluster(bar, bytes);  // the copy's bytes + own lo half
          }
        }
      }
      return __shfl_sync(0xffffffffu, p_ok, 0) != 0;
    };
    // accumulator rows of this thread: TMEM lane 32 q + lane of slot `slot`
    auto trow_of = [&](int slot) -> uint32_t {
      return tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(slot * 256);
    };

    // input layer (FP32): a_1 = tanh(W_0 z + b_0) for the rows of this CTA's
    // blocks (j = 2 m + rank) and the nodes of this warp half; d_1 to the
    // scratch, own half into X (forward layout), the peer's half staged
    auto input_layer = [&](int tile, int it_) -> bool {
      const int node0 = tile * NPC, nb = 24 * half;
      mark(it_, n_gemm, 2);
      // W_0 row and bias of M tile 0, before the waits
      float w[NZ], bi;
      {
        const int i = 128 * (int)rank + 32 * q + lane;
#pragma unroll
        for (int jj = 0; jj < NZ; ++jj) w[jj] = a.W0[(size_t)jj * HP + i];
        bi = a.b0[i];
      }
      if (!wwait(z_free, zr_ph ^ 1u)) return false;  // every warp done with the last z
      zr_ph ^= 1u;
#pragma unroll
      for (int h = 0; h < 3; ++h)
        if (et + 256 * h < NZV) zbuf[((et + 256 * h) / NZ) * ZS + (et + 256 * h) % NZ] = zpref[h];
      __syncwarp();
      if (lane == 0) mbar_arrive(z_full);
      if (!wwait(z_full, zf_par)) return false;
      zf_par ^= 1u;
      if (it_ > 0) {
        // every warp has read the previous tile's d (its backward pass)
        if (!wwait(bwd_done, bd_par)) return false;
        bd_par ^= 1u;
        // the previous tile's W_0' MMAs have read every block (both layouts
        // share the buffer, so all blocks before any is rewritten)
        for (int jj = 0; jj < nblk; ++jj)
          if (!wwait(xfree(jj), (uint32_t)(n_gemm * it_ - 1) & 1u)) return false;
      }
      for (int m = 0; m < n_mt2; ++m) {
        const int j = 2 * m + (int)rank;
        const int i = 128 * j + 32 * q + lane;
        float av[24];
#pragma unroll
        for (int g8 = 0; g8 < 3; ++g8) dot17_x8(w, zbuf, nb + 8 * g8, NPC, bi, av + 8 * g8);
        if (m + 1 < n_mt2) {  // the next M tile's W_0 row and bias
#pragma unroll
          for (int jj = 0; jj < NZ; ++jj) w[jj] = a.W0[(size_t)jj * HP + i + 256];
          bi = a.b0[i + 256];
        }
        tanh_batch<24>(av);
        act_finish<24>(av, dptr(0, i) + (size_t)nb * HP, HP, min(NPC, a.n_nodes - node0) - nb, NPC - nb);
        uint32_t own[12], peer[12];
#pragma unroll
        for (int p = 0; p < 12; ++p) {
          uint32_t hv, lv;
          split2(av[2 * p], av[2 * p + 1], hv, lv);
          own[p] = lo_local ? lv : hv;
          peer[p] = lo_local ? hv : lv;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
          *reinterpret_cast<uint4*>(X + xoff_n(R2_CF, i, nb + 8 * c)) =
              make_uint4(own[4 * c], own[4 * c + 1], own[4 * c + 2], own[4 * c + 3]);
        if (!wait_staging()) return false;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          *reinterpret_cast<uint4*>(S + xoff_n(R2_CF, i & 127, nb + 8 * c)) =
              make_uint4(peer[4 * c], peer[4 * c + 1], peer[4 * c + 2], peer[4 * c + 3]);
        if (!block_end(j, 128u * R2_CF * 2u, 0u)) return false;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(z_free);
      mark_end(it_, n_gemm);
      return true;
    };

    // forward hidden layer g: a = tanh(acc + b) for the nodes of this half,
    // d to the scratch, own half into X, the peer's half staged
    auto fwd_layer = [&](int it_, int g, int node0) -> bool {
      mark(it_, g, 2);
      for (int m = 0; m < n_mt2; ++m) {
        stamp(it_, g, m, 0);
        const float bi = a.bias[(size_t)g * HP + 128 * (2 * m + (int)rank) + 32 * q + lane];  // before the waits
        if (!wwait(acc_full(m), (acc_par >> m) & 1u)) return false;
        acc_par ^= 1u << m;
        tc_fence_after();
        stamp(it_, g, m, 1);
        const int j = 2 * m + (int)rank;  // the block this CTA's rows produce
        // written to the forward half GEMM g does not read (its last reader,
        // GEMM g - 1, completed before GEMM g's accumulator)
        const uint32_t xo = (uint32_t)((g + 1) & 1) * (xbytes / 2u);
        stamp(it_, g, m, 2);
        const int i = 128 * j + 32 * q + lane;
        const int nb = 24 * half, c0 = 16 * half;  // nodes nb..nb+23 lie in columns c0..c0+31
        const uint32_t tr_ = trow_of(m);
        float v[32], w[32];
        tmem_ld16(tr_ + c0, v);
        tmem_ld16(tr_ + c0 + 16, v + 16);
        tmem_ld16(tr_ + R2_CF + c0, w);
        tmem_ld16(tr_ + R2_CF + c0 + 16, w + 16);
        tmem_wait_ld();
        // the accumulator slot is free once its loads completed
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive_cluster_relaxed(tf0 + 8u * m);
        stamp(it_, g, m, 3);
        // in batched phases over the 24 nodes (independent chains side by
        // side): node nb + t is accumulator column t (half 0) or 8 + t
        float av[24];
#pragma unroll
        for (int t = 0; t < 24; ++t) av[t] = (half ? v[8 + t] + w[8 + t] : v[t] + w[t]) + bi;
        tanh_batch<24>(av);
        act_finish<24>(av, dptr(g + 1, i) + (size_t)nb * HP, HP, min(NPC, a.n_nodes - node0) - nb, NPC - nb);
        uint32_t own[12], peer[12];
#pragma unroll
        for (int p = 0; p < 12; ++p) {
          uint32_t hv, lv;
          split2(av[2 * p], av[2 * p + 1], hv, lv);
          own[p] = lo_local ? lv : hv;
          peer[p] = lo_local ? hv : lv;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
          *reinterpret_cast<uint4*>(X + xo + xoff_n(R2_CF, i, nb + 8 * c)) =
              make_uint4(own[4 * c], own[4 * c + 1], own[4 * c + 2], own[4 * c + 3]);
        stamp(it_, g, m, 4);
        if (!wait_staging()) return false;
        stamp(it_, g, m, 5);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          *reinterpret_cast<uint4*>(S + xoff_n(R2_CF, i & 127, nb + 8 * c)) =
              make_uint4(peer[4 * c], peer[4 * c + 1], peer[4 * c + 2], peer[4 * c + 3]);
        stamp(it_, g, m, 6);
        if (!block_end(j, 128u * R2_CF * 2u, xo)) return false;
        stamp(it_, g, m, 7);
      }
      mark_end(it_, g);
      return true;
    };

    // output layer: f_D from rank 0's TMEM lanes 0..2 of slot 1 (value
    // columns n hi, R2_CF + n lo)
    auto out_layer = [&](int it_, int node0) -> bool {
      mark(it_, nh, 2);
      if (!wwait(acc_full(1), (acc_par >> 1) & 1u)) return false;
      acc_par ^= 2u;
      tc_fence_after();
      if (rank == 0 && q == 0) {
        const int nb = 24 * half, c0 = 16 * half;
        float v[32], w[32];
        const uint32_t tr_ = tmem + 256u;
        tmem_ld16(tr_ + c0, v);
        tmem_ld16(tr_ + c0 + 16, v + 16);
        tmem_ld16(tr_ + R2_CF + c0, w);
        tmem_ld16(tr_ + R2_CF + c0 + 16, w + 16);
        tmem_wait_ld();
        const float bo = lane < NO ? a.bias[(size_t)nh * HP + lane] : 0.0f;
#pragma unroll
        for (int n2 = 0; n2 < 24; ++n2) {
          const int n = nb + n2, node = node0 + n;
          const float acc = half ? v[8 + n2] + w[8 + n2] : v[n2] + w[n2];
          if (n < NPC && lane < NO && node < a.n_nodes) a.fD[(size_t)node * NO + lane] = acc + bo;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_cluster_relaxed(tf0 + 8u);
      mark_end(it_, nh);
      return true;
    };

    // 16 backward columns cl0.. of this half (3 n + i) of row i: own half
    // into X, the peer's half into peer[8 c2 ..]
    auto bwd_chunk = [&](int i, int c2, const float (&v)[16], uint32_t (&peer)[32]) {
      const int cb = 64 * half + 16 * c2;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t own[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          uint32_t hv, lv;
          split2(v[8 * c + 2 * p], v[8 * c + 2 * p + 1], hv, lv);
          own[p] = lo_local ? lv : hv;
          peer[8 * c2 + 4 * c + p] = lo_local ? hv : lv;
        }
        *reinterpret_cast<uint4*>(X + xoff_n(R2_CB, i, cb + 8 * c)) = make_uint4(own[0], own[1], own[2], own[3]);
      }
    };
    // the staged peer half of row i, then the block push
    auto bwd_flush = [&](int j, int i, const uint32_t (&peer)[32]) -> bool {
      if (!wait_staging()) return false;
      const int cb = 64 * half;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<uint4*>(S + xoff_n(R2_CB, i & 127, cb + 8 * c)) =
            make_uint4(peer[4 * c], peer[4 * c + 1], peer[4 * c + 2], peer[4 * c + 3]);
      return block_end(j, 128u * R2_CB * 2u, 0u);
    };
    // d of the 22 nodes whose adjoint columns this half holds (node n0 + k);
    // column c of the half is component (c + half) % 3 of node n0 + (c + half) / 3
    const int n0 = (64 * half) / 3;  // 0 or 21
    auto load_d = [&](int layer, int i, float (&dd)[22]) {
      const float* dr = dptr(layer, i);
#pragma unroll
      for (int k = 0; k < 22; ++k) dd[k] = n0 + k < NPC ? dr[(size_t)(n0 + k) * HP] : 0.0f;
    };

    // adjoints of the last hidden layer, D_L = d_L (.) W_L' (no accumulator,
    // no exchange): this CTA writes its own half (hi or lo) of the 64 columns
    // of this warp half for every row; blocks in the MMAs' order (1, 0, 3, 2)
    auto dl_init = [&](int it_) -> bool {
      mark(it_, n_gemm, 0);
      const int cb = 64 * half;
      // W_L columns of this thread's rows in every block (MMA order 1, 0, 3, 2)
      float wl[NB][3];
#pragma unroll
      for (int jb = 0; jb < NB; ++jb)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          wl[jb][k] = jb < nblk ? a.WL[(size_t)k * HP + 128 * (jb ^ 1) + 32 * q + lane] : 0.0f;
      // every epilogue warp of both CTAs has written its d_L of this tile
      stamp(it_, nh, 0, 0);
      __syncwarp();
      if (lane == 0) {
        arrive_cluster(dr0);
        arrive_cluster(dr1);
      }
      {
        int w_ok = 0;
        if (lane == 0) w_ok = mbar_wait_cl(d_ready, dr_par, abort_flag, a.err);
        if (!__shfl_sync(0xffffffffu, w_ok, 0)) return false;
        __syncwarp();
        dr_par ^= 1u;
      }
      stamp(it_, nh, 0, 1);
      float dn[22];  // d of the next block, loaded one block ahead
      load_d(nh, 128 * 1 + 32 * q + lane, dn);
      for (int jb = 0; jb < nblk; ++jb) {
        const int j = jb ^ 1;
        const int i = 128 * j + 32 * q + lane;
        float dd[22];
#pragma unroll
        for (int k = 0; k < 22; ++k) dd[k] = dn[k];
        if (jb + 1 < nblk) load_d(nh, 128 * ((jb + 1) ^ 1) + 32 * q + lane, dn);
        float wlj[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) wlj[k] = jb == 0 ? wl[0][k] : jb == 1 ? wl[1][k] : jb == 2 ? wl[2][k] : wl[3][k];
        // the output layer's MMAs have read every block (the layouts switch)
        if (jb == 0) {
          for (int jj = 0; jj < nblk; ++jj)
            if (!wwait(xfree(jj), xfree_par(it_, nh))) return false;
          stamp(it_, nh, 0, 2);
        }
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
          uint32_t own[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int c = 8 * c2 + 2 * p + h;  // column within the half
              const float p0 = dd[c / 3] * wlj[c % 3];                             // half 0
              const float p1 = c < 62 ? dd[(c + 1) / 3] * wlj[(c + 1) % 3] : 0.0f;  // half 1
              v2[h] = half ? p1 : p0;
            }
            uint32_t hv, lv;
            split2(v2[0], v2[1], hv, lv);
            own[p] = lo_local ? lv : hv;
          }
          *reinterpret_cast<uint4*>(X + xoff_n(R2_CB, i, cb + 8 * c2)) = make_uint4(own[0], own[1], own[2], own[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (rank == 0)
            mbar_arrive(xin(j));
          else
            arrive_cluster(xi0 + 8u * j);
        }
        stamp(it_, nh, 0, 3 + jb);
      }
      mark(it_, n_gemm, 1);
      ew = 0;
      return true;
    };

    // backward hidden layer g (l = 2 nh + 1 - g): D_l = d_l (.) (W_l' D_{l+1})
    auto bwd_layer = [&](int it_, int g) -> bool {
      const int l = 2 * nh + 1 - g;
      mark(it_, g, 2);
      for (int m = 0; m < n_mt2; ++m) {
        const int j = 2 * m + (int)rank;
        const int i = 128 * j + 32 * q + lane;
        stamp(it_, g, m, 0);
        float dd[22];
        load_d(l - 1, i, dd);  // issued before the waits
        if (!wwait(acc_full(m), (acc_par >> m) & 1u)) return false;
        acc_par ^= 1u << m;
        tc_fence_after();
        stamp(it_, g, m, 1);
        if (!wwait(xfree(j), xfree_par(it_, g))) return false;
        stamp(it_, g, m, 2);
        const uint32_t tr_ = trow_of(m) + (uint32_t)(64 * half);
        uint32_t peer[32];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float h16[16], l16[16];
          tmem_ld16(tr_ + 16 * c, h16);
          tmem_ld16(tr_ + R2_CB + 16 * c, l16);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int cl = 16 * c + k;  // column within the half
            const float dn = half ? (cl < 62 ? dd[(cl + 1) / 3] : 0.0f) : dd[cl / 3];
            h16[k] = (h16[k] + l16[k]) * dn;
          }
          bwd_chunk(i, c, h16, peer);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive_cluster_relaxed(tf0 + 8u * m);
        stamp(it_, g, m, 3);
        if (!bwd_flush(j, i, peer)) return false;
        stamp(it_, g, m, 7);
      }
      mark_end(it_, g);
      return true;
    };

    // J_D = W_0' D_1 from rank 0's TMEM lanes 0..16 of slot 1
    auto jd_readout = [&](int it_, int node0) -> bool {
      mark(it_, n_gemm - 1, 2);
      if (!wwait(acc_full(1), (acc_par >> 1) & 1u)) return false;
      acc_par ^= 2u;
      tc_fence_after();
      if (rank == 0 && q == 0) {
        const uint32_t tr_ = tmem + 256u + (uint32_t)(64 * half);
        // column cc = 3 n + i is row (node0 + n) * 3 + i of J_D: entry
        // (3 node0 + cc) * 17 + lane; columns of real nodes end at `lim`
        const int lim = 3 * min(NPC, a.n_nodes - node0) - 64 * half;
        float* jrow = a.JD + ((size_t)node0 * NO + 64 * half) * NZ + lane;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float h16[16], l16[16];
          tmem_ld16(tr_ + 16 * c, h16);
          tmem_ld16(tr_ + R2_CB + 16 * c, l16);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (16 * c + k < lim && lane < NZ) jrow[(16 * c + k) * NZ] = h16[k] + l16[k];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_cluster_relaxed(tf0 + 8u);
      mark_end(it_, n_gemm - 1);
      return true;
    };

    int it = 0;
    if (pair < n_tiles) ok = input_layer(pair, 0);
    for (int tile = pair; tile < n_tiles && ok; tile += n_pairs, ++it) {
      const int node0 = tile * NPC;
      for (int g = 0; g < nh && ok; ++g) ok = fwd_layer(it, g, node0);
      // the last-layer adjoints while the output layer's MMAs run; f_D after
      // them (the first backward GEMM's second M tile reuses that slot)
      if (ok) ok = dl_init(it);
      if (ok) ok = out_layer(it, node0);
      if (ok && nh == 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bwd_done);
      }
      for (int g = nh + 1; g <= 2 * nh && ok; ++g) {
        ok = bwd_layer(it, g);
        if (ok && g == 2 * nh) {
          __syncwarp();
          if (lane == 0) mbar_arrive(bwd_done);
        }
      }
      if (!ok) break;
      // J_D, then the next tile's input layer (its first GEMM's second M
      // tile reuses the accumulator slot of W_0')
      const int nt = tile + n_pairs;
      if (nt < n_tiles) prefetch_z(nt);
      if (!(ok = jd_readout(it, node0))) break;
      if (nt < n_tiles && !(ok = input_layer(nt, it + 1))) break;
    }
    // tail: the last W_0' GEMM's release of every block (its commit reaches
    // both CTAs)
    if (ok && it > 0)
      for (int j = 0; j < nblk && ok; ++j) ok = wwait(xfree(j), (uint32_t)(n_gemm * it - 1) & 1u);
  }

  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                 : "memory");
  }
}

}  // namespace

// shared memory of the pair reverse-mode kernel with `stages` weight stages
size_t mlp_rev2_smem(int HP, int stages) {
  const int nbar = 2 * stages + 2 * 2 + 4 * 4 + 6;
  return 1024 + (size_t)R2_CB * HP * 2 + R2_SBYTES + (size_t)stages * WT_BYTES + 8 * nbar + 16 +
         (size_t)R2_NPC * ZS * 4;
}

cudaError_t mlp_rev2_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  TcNet& tc = ctx->net.tc;
  Rev2Args a;
  a.x = x;
  a.u = u;
  a.node_inst = ctx->lay.node_inst;
  a.n_nodes = ctx->lay.n_nodes;
  a.W0 = tc.W0;
  a.b0 = tc.b0;
  a.bias = tc.bias;
  a.WL = tc.WL32;
  a.HP = tc.h_pad;
  a.n_hidden_mm = tc.n_mm;
  a.tmem_cols = (uint32_t)tc.tmem_cols;
  a.fD = fD;
  a.JD = JD;
  a.dscr = tc.dscr;
  a.err = tc.err;
  a.trace = tc.trace;
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(tc.tmapR_bytes);
  void* args[] = {(void*)map, (void*)&a};
  const int n_tiles = (a.n_nodes + R2_NPC - 1) / R2_NPC;
  // pairs: the scratch has n_sm / 2 pair slots of R2_NPC nodes
  dim3 grid(2 * std::min(n_tiles, std::max(1, tc.n_sm / 2)));
  return cudaLaunchKernel(tc.fn, grid, dim3(R2_THREADS), args, tc.smem, ctx->stream);
}

// kernel entry of the pair reverse-mode shape with `stages` weight stages, or null
const void* mlp_rev2_fn(int npc, int stages) {
  if (npc != R2_NPC) return nullptr;
  if (stages == 3) return (const void*)&mlp_rev2_kernel<3>;
  if (stages == 6) return (const void*)&mlp_rev2_kernel<6>;
  return nullptr;
}

}  // namespace rtn

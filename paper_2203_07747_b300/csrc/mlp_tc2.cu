// mlp_tc2.cu -- (a1) the split-BF16 network kernel on CTA pairs.
//
// Same computation as mlp_tc.cu (forward-mode value + 17 tangents per node,
// Sec. III-A Eq. 4), for the case where one SM cannot hold enough node
// columns: a cluster of two CTAs runs tcgen05.mma with cta_group::2 and
// M = 256 output neurons per instruction.
//   * rank 0 holds X_hi, rank 1 holds X_lo of the same C node columns (both
//     N-major, same shared-memory offset); one MMA of N = 2C reads X_hi from
//     rank 0 and X_lo from rank 1 and writes W X_hi | W X_lo into the
//     accumulator of each CTA, whose tensor memory holds that CTA's 128 of
//     the 256 output rows;
//   * each CTA streams its 128 weight rows of every 256-row tile by TMA; both
//     halves complete on rank 0's stage barrier (cta_group::2 copies), which
//     expects the bytes of the pair;
//   * rank 0's thread issues every MMA; the commits arrive on both CTAs.
// Rows of X are tracked in 128-row blocks; block j is produced by the CTA
// whose accumulator holds those rows (rank j % 2).  The producer adds the two
// accumulator halves, applies tanh and tanh', writes its own half of the
// block (hi on rank 0, lo on rank 1) straight into its X and the peer's half
// into a local staging buffer, and one thread pushes the staged 128-row block
// to the peer with a single bulk copy that completes on a barrier by byte
// count.  The epilogue warps therefore never wait on remote stores.  A copy
// has read its staging block once its destination barrier completed: the
// thread that sees that completion frees the producer's staging block
// (s_free):
//   * block j odd (rank 1): the copy lands in rank 0's X and completes on
//     rank 0's xready[j]; the same arrival (release, cluster scope) publishes
//     rank 1's own half; rank 0's exchange warp sees xready[j] complete and
//     frees rank 1's staging block;
//   * block j even (rank 0): the copy lands in rank 1's X and completes on
//     rank 1's lo_in[j]; rank 1's exchange warp forwards it to xready[j]
//     and frees rank 0's staging block.
// The exchange warps (warp 10 of each CTA) wait on nothing the MMA issuer
// or the epilogue must do first, so a staging block is freed however far the
// MMA issuer has got (it may itself wait on the epilogue that needs it).
// The input layer (FP32, 17 inputs) needs no exchange: both CTAs compute
// every row and keep their own half of the columns; all 16 epilogue warps
// arrive on rank 0's xin[j].  The notice that the MMAs have read block j
// (xfree) reaches both CTAs, and every wait on it names its completion by
// the layer count (one completion per layer).
// Every wait is bounded (RTN_E_TIMEOUT in the device flag).  After the pair
// allocates tensor memory it checks that both CTAs received the same address;
// if not it records RTN_E_UNSUPPORTED and does no work.
#include <algorithm>
#include <type_traits>

#include "tc_pair.cuh"

namespace rtn {
namespace {

// the peer's half of nodes N0..N1-1 for one row, held in registers until
// the staging block is free (hi halves on rank 1, lo halves on rank 0)
template <int NPC, int C, int N0, int N1>
struct PeerHalf {
  static constexpr int END = N1;
  uint4 t[N1 - N0][2];
  uint32_t ve[N1 - N0];  // value (bits 0..15) and 17th tangent (16..31)
  __device__ __forceinline__ void put(int n, const NodeOut& o, bool lo_local) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      t[n - N0][h] = lo_local ? make_uint4(o.th[4 * h], o.th[4 * h + 1], o.th[4 * h + 2], o.th[4 * h + 3])
                              : make_uint4(o.tl[4 * h], o.tl[4 * h + 1], o.tl[4 * h + 2], o.tl[4 * h + 3]);
    ve[n - N0] = lo_local ? ((o.v & 0xffffu) | (o.e << 16)) : ((o.v >> 16) | (o.e & 0xffff0000u));
  }
  // row k of the 128-row block into the staging block S
  __device__ __forceinline__ void flush(uint8_t* S, int k) const {
    const int ks = k & 127;
#pragma unroll
    for (int n = N0; n < N1; ++n) {
#pragma unroll
      for (int h = 0; h < 2; ++h) *reinterpret_cast<uint4*>(S + xoff<C>(ks, 16 * n + 8 * h)) = t[n - N0][h];
      *reinterpret_cast<uint16_t*>(S + xoff<C>(ks, 16 * NPC + n)) = (uint16_t)(ve[n - N0] & 0xffffu);
      *reinterpret_cast<uint16_t*>(S + xoff<C>(ks, 17 * NPC + n)) = (uint16_t)(ve[n - N0] >> 16);
    }
  }
};

// one node's row-k results, this CTA's half only
template <int NPC, int C>
__device__ __forceinline__ void node_store_own(uint8_t* X, bool lo_local, int k, int n, const NodeOut& o) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = 16 * n + 8 * h;
    const uint4 hv = make_uint4(o.th[4 * h], o.th[4 * h + 1], o.th[4 * h + 2], o.th[4 * h + 3]);
    const uint4 lv = make_uint4(o.tl[4 * h], o.tl[4 * h + 1], o.tl[4 * h + 2], o.tl[4 * h + 3]);
    *reinterpret_cast<uint4*>(X + xoff<C>(k, c)) = lo_local ? lv : hv;
  }
  *reinterpret_cast<uint16_t*>(X + xoff<C>(k, 16 * NPC + n)) =
      lo_local ? (uint16_t)(o.v >> 16) : (uint16_t)(o.v & 0xffffu);
  *reinterpret_cast<uint16_t*>(X + xoff<C>(k, 17 * NPC + n)) =
      lo_local ? (uint16_t)(o.e >> 16) : (uint16_t)(o.e & 0xffffu);
}

// warps 0..9 as in mlp_tc.cu, warp 10: activation exchange
constexpr int THREADS2 = THREADS + 32;

template <int NPC, int STAGES>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS2, 1)
    mlp_tc2_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  constexpr int C = Cols<NPC>::C, TAIL = Cols<NPC>::TAIL, HALF = (NPC + 1) / 2;
  constexpr int NMMA = 2 * C;  // hi columns (rank 0) then lo columns (rank 1)
  static_assert(NMMA % 16 == 0 && NMMA <= 256, "MMA N");
  constexpr int NZV = NPC * NZ;
  constexpr int MT = 2, NB = 4;  // <= 2 tiles of 256 rows, <= 4 blocks of 128 rows
  constexpr uint32_t SBYTES = 128u * C * 2u;  // one 128-row block of one CTA's columns
  extern __shared__ uint8_t smem_raw[];
  const uint32_t rank = cluster_rank();
  const int HP = a.HP, n_mt2 = HP / 256, nkb = HP / 64, nblk = HP / 128;
  const int nh = a.n_hidden_mm, n_layers = nh + 1;
  const int n_tiles = (a.n_nodes + NPC - 1) / NPC;
  const int pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t sbase = sraw + pad;
  const uint32_t xbytes = (uint32_t)C * HP * 2u;
  uint8_t* X = sm;                                  // X_hi (rank 0) / X_lo (rank 1)
  uint8_t* S = sm + xbytes;                         // staging block for the peer's half
  const uint32_t x_s = sbase, s_s = sbase + xbytes;
  const uint32_t x_rem = mapa(x_s, rank ^ 1u);      // the peer's X
  const bool lo_local = rank == 1;
  const uint32_t w_s = sbase + xbytes + SBYTES;
  uint8_t* tail_area = sm + xbytes + SBYTES + STAGES * WT_BYTES;
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
  constexpr int NBAR = 2 * STAGES + 2 * MT + 4 * NB + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail_area + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* zbuf = reinterpret_cast<float*>(tail_area + 8 * NBAR + 16);

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
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero this CTA's X (padding columns stay 0) and S before the peer may copy into X
  for (uint32_t o = threadIdx.x * 16u; o < xbytes + SBYTES; o += THREADS2 * 16u)
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
    // issues): this CTA's 128 rows of each 256-row tile
    if (lane == 0)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    {
      const uint32_t full0 = mapa(full_bar(0), 0);  // stage barriers of rank 0
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs)
        for (int l = 0; l < n_layers && ok; ++l) {
          const int mts = (l < nh) ? n_mt2 : 1;
          for (int m = 0; m < mts && ok; ++m)
            for (int kb = 0; kb < nkb && ok; ++kb) {
              if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err))) break;
              if (elect_one()) {
                // the output layer's rows 128..255 (rank 1's half) are padding
                // whose products land in accumulator rows nobody reads: not loaded
                const bool load = l < nh || rank == 0;
                if (rank == 0) mbar_expect_tx(full_bar(s), (l < nh ? 2 : 1) * WT_BYTES);
                const int kk = kb ^ 2;  // K order of the MMAs (blocks 1, 0, 3, 2)
                if (load) {
#pragma unroll
                  for (int bx = 0; bx < W_BOXES; ++bx)
                    tma_load_2d_pair(w_s + s * WT_BYTES + bx * 4096u, &tmap, kk * 64 + bx * W_BOX_K,
                                     l * HP + m * 256 + (int)rank * 128, full0 + 8u * s);
                }
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
      constexpr uint32_t idesc = idesc_bf16(256, NMMA) | (1u << 16);  // B is N-major
      const uint32_t lbo = C * 16u;
      int s = 0;
      uint32_t ph = 0, used = 0, tf_par = 0, xr_par = 0, xi_par = 0;
      bool ok = true;
      int it = 0;
      WaitClock wc(a.trace != nullptr && blockIdx.x == 0);
      long long w_odd = 0, w_even = 0;
      const bool tl = RTN_TRACE && lane == 0;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs, ++it)
        for (int l = 0; l < n_layers && ok; ++l) {
          if (tl) trace(a, it, l, n_layers, 0);
          long long w_x = 0, w_w = 0, w_t = 0;
          const int mts = (l < nh) ? n_mt2 : 1;
          for (int m = 0; m < mts && ok; ++m) {
            // accumulator slot: M tile m; the output layer uses slot 1 so that
            // the next tile's first M tile need not wait for its read-out
            const int slot = (l < nh) ? m : 1;
            if (used & (1u << slot)) {
              wc.start();
              ok = mbar_wait_cl_warp(tmem_free(slot), (tf_par >> slot) & 1u, abort_flag, a.err);
              wc.stop(w_t);
              if (!ok) break;
              tf_par ^= 1u << slot;
            }
            used |= 1u << slot;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(slot * NMMA);
            for (int kb = 0; kb < nkb && ok; ++kb) {
              // K is summed in the order blocks 1, 0, 3, 2: each odd block
              // (copied straight into rank 0) is used while the even block
              // before it is still being relayed
              const int kk = kb ^ 2, j = kk >> 1;
              if (m == 0 && (kb & 1) == 0) {
                long long w0 = w_x;
                wc.start();
                if (l == 0) {  // the input layer's blocks
                  ok = mbar_wait_cl_warp(xin(j), (xi_par >> j) & 1u, abort_flag, a.err);
                  xi_par ^= 1u << j;
                } else {
                  ok = mbar_wait_cl_warp(xready(j), (xr_par >> j) & 1u, abort_flag, a.err);
                  xr_par ^= 1u << j;
                }
                wc.stop(w_x);
                ((j & 1) ? w_odd : w_even) += w_x - w0;
                if (!ok) break;
                tc_fence_after();
              }
              wc.start();
              ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err);
              wc.stop(w_w);
              if (!ok) break;
              tc_fence_after();
              const uint32_t as = w_s + s * WT_BYTES;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t bo = (uint32_t)(kk * 4 + ks) * 2u * lbo;
                mma2_bf16(d, wdesc(as, ks), xdesc(x_s + bo, lbo), idesc, (kb | ks) != 0);
              }
              commit2(empty_bar(s), 3);
              if (++s == STAGES) { s = 0; ph ^= 1u; }
              // the layer's last M tile has read block j: its producer may rewrite it
              if (m == mts - 1 && (kb & 1)) commit2(xfree(j), 3);
            }
            if (ok) commit2(acc_full(slot), 3);
          }
          if (tl) {
            trace(a, it, l, n_layers, 1);
            trace_put(a, it, l, n_layers, 4, w_x);
            trace_put(a, it, l, n_layers, 5, w_w);
            trace_put(a, it, l, n_layers, 6, w_t);
          }
          if (l == n_layers - 1) {
            if (tl) {
              trace_put(a, it, n_layers, n_layers, 6, w_odd);
              trace_put(a, it, n_layers, n_layers, 7, w_even);
            }
            w_odd = w_even = 0;
          }
        }
    }
  } else if (run && warp == THREADS / 32) {
    if (lane == 0) {
      // ---------------- exchange warp: hidden-layer outputs, blocks in the
      // order their producers publish them
      const uint32_t xr0 = mapa(xready(0), 0);
      const uint32_t sfree_peer = mapa(s_free, rank ^ 1u);
      uint32_t par = 0;
      bool ok = true;
      for (int tile = pair; tile < n_tiles && ok; tile += n_pairs)
        for (int l = 0; l < nh && ok; ++l)
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
    const int e = warp - 2;
    const int q = warp & 3;
    const int half = e >> 2;
    const int et = threadIdx.x - 64;
    const bool elected = (e == 0 && lane == 0);  // publishes each block
    float zpref = (et < NZV) ? load_z(a, pair * NPC + et / NZ, et % NZ) : 0.0f;
    uint32_t acc_par = 0, sf_ph = 0, ss_par = 0, zf_par = 0, zr_ph = 0;
    bool ok = true;
    const bool tr = RTN_TRACE && (rank == 0 && e == 0 && lane == 0);
    const uint32_t tf0 = mapa(tmem_free(0), 0);
    const uint32_t xr0 = mapa(xready(0), 0), lo1 = mapa(lo_in(0), 1), xi0 = mapa(xin(0), 0);
    // xfree[j] completes once per MMA layer: completion c (from 1) of this
    // pair's tile it, layer l is c = n_layers it + l + 1; wait parity (c-1)&1
    auto xfree_par = [&](int it_, int l) -> uint32_t { return (uint32_t)(n_layers * it_ + l) & 1u; };
    long long epi_wait = 0, t_work = 0, t_sfull = 0, t_copy = 0;
    WaitClock ewc(tr && a.trace != nullptr && blockIdx.x == 0);

    auto wwait = [&](uint32_t bar, uint32_t par) -> bool {
      int w_ok = 0;
      ewc.start();
      if (lane == 0) w_ok = mbar_wait(bar, par, abort_flag, a.err);
      ewc.stop(epi_wait);
      return __shfl_sync(0xffffffffu, w_ok, 0) != 0;
    };

    // before the staging block is rewritten: the previous copy has landed
    auto wait_staging = [&]() -> bool {
      if (!wwait(s_free, sf_ph ^ 1u)) return false;
      sf_ph ^= 1u;
      return true;
    };

    // after every warp wrote its rows of block j: publish own half, push the
    // peer's half
    auto block_end = [&](int j) -> bool {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(s_full);
      int p_ok = 1;
      if (elected) {
        ewc.start();
        p_ok = mbar_wait(s_full, ss_par, abort_flag, a.err);
        ewc.stop(t_sfull);
        ss_par ^= 1u;
        ewc.start();
        if (p_ok) {
          const uint32_t bar = (rank == 0 ? lo1 : xr0) + 8u * j;
#pragma unroll
          for (int c = 0; c < 4; ++c)  // four copies in flight, issued first
            bulk_copy_to_peer(x_rem + (uint32_t)j * SBYTES + c * (SBYTES / 4), s_s + c * (SBYTES / 4),
                              SBYTES / 4, bar);
          if (rank == 0) {
            mbar_arrive(xready(j));                             // own hi half
            arrive_expect_tx_cluster_relaxed(bar, SBYTES);      // the copy's bytes
          } else {
            arrive_expect_tx_cluster(bar, SBYTES);  // the copy's bytes + own lo half
          }
        }
        ewc.stop(t_copy);
      }
      return __shfl_sync(0xffffffffu, p_ok, 0) != 0;
    };

    // input layer (FP32): this CTA computes every row and keeps its own
    // half of the columns; blocks in the order the MMAs read them (1, 0, 3, 2)
    auto input_layer = [&](int tile, int it_) -> bool {
      const int node0 = tile * NPC;
      if (!wwait(z_free, zr_ph ^ 1u)) return false;  // every warp done with the last z
      zr_ph ^= 1u;
      if (et < NZV) zbuf[et] = zpref;
      __syncwarp();
      if (lane == 0) mbar_arrive(z_full);
      if (!wwait(z_full, zf_par)) return false;
      zf_par ^= 1u;
      if (tr) trace(a, it_, n_layers, n_layers, 0);
      const int hh = et >> 7;
      for (int jb = 0; jb < nblk; ++jb) {
        const int j = jb ^ 1;
        const int i = 128 * j + (et & 127);
        float w[NZ];
#pragma unroll
        for (int jj = 0; jj < NZ; ++jj) w[jj] = a.W0[(size_t)jj * HP + i];
        const float bi = a.b0[i];
        // the previous tile's output layer has read block j
        if (it_ > 0 && !wwait(xfree(j), (uint32_t)(n_layers * it_ - 1) & 1u)) return false;
#pragma unroll
        for (int n = 0; n < NPC; ++n) {
          if ((n < HALF) != (hh == 0)) continue;
          float sacc = bi;
#pragma unroll
          for (int jj = 0; jj < NZ; ++jj) sacc = fmaf(w[jj], zbuf[n * NZ + jj], sacc);
          const bool real = node0 + n < a.n_nodes;
          const float av = real ? tanh_tc(sacc) : 0.0f, d = real ? 1.0f - av * av : 0.0f;
          NodeOut o;
          node_pack<1>(av, d, w, w[16], o);
          node_store_own<NPC, C>(X, lo_local, i, n, o);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (rank == 0)
            mbar_arrive(xin(j));
          else
            arrive_cluster(xi0 + 8u * j);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(z_free);
      if (tr) trace(a, it_, n_layers, n_layers, 1);
      return true;
    };

    int it = 0;
    if (pair < n_tiles) ok = input_layer(pair, 0);
    for (int tile = pair; tile < n_tiles && ok; tile += n_pairs, ++it) {
      const int node0 = tile * NPC;
      for (int l = 0; l < nh && ok; ++l) {
        for (int m = 0; m < n_mt2; ++m) {
          if (!(ok = wwait(acc_full(m), (acc_par >> m) & 1u))) break;
          acc_par ^= 1u << m;
          if (tr && m == 0) trace(a, it, l, n_layers, 2);
          tc_fence_after();
          const int j = 2 * m + (int)rank;  // the block this CTA's rows produce
          // the MMAs of layer l have read block j's old contents
          if (!(ok = wwait(xfree(j), xfree_par(it, l)))) break;
          ewc.start();
          const int i = 128 * j + 32 * q + lane;
          const float bi = a.bias[(size_t)l * HP + i];
          const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * NMMA);
          // own half into X now, the peer's half once the staging block is free
          auto run_nodes = [&](auto& peer, auto n0) -> bool {
            auto store = [&](int n, const NodeOut& o) {
              node_store_own<NPC, C>(X, lo_local, i, n, o);
              peer.put(n, o, lo_local);
            };
            epilogue_nodes<NPC, C, 2, decltype(n0)::value, std::remove_reference_t<decltype(peer)>::END>(
                trow, bi, store);
            // the accumulator tile is free once its loads completed
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_cluster_relaxed(tf0 + 8u * m);
            if (!wait_staging()) return false;
            peer.flush(S, i);
            return true;
          };
          if (half == 0) {
            PeerHalf<NPC, C, 0, HALF> peer;
            ok = run_nodes(peer, std::integral_constant<int, 0>());
          } else {
            PeerHalf<NPC, C, HALF, NPC> peer;
            ok = run_nodes(peer, std::integral_constant<int, HALF>());
          }
          ewc.stop(t_work);
          if (!ok) break;
          if (!(ok = block_end(j))) break;
        }
        if (tr) {
          trace(a, it, l, n_layers, 3);
          trace_put(a, it, l, n_layers, 7, epi_wait);
          epi_wait = 0;
        }
      }
      if (!ok) break;
      if (tr) {
        trace_put(a, it, n_layers, n_layers, 2, t_work);
        trace_put(a, it, n_layers, n_layers, 3, t_sfull);
        trace_put(a, it, n_layers, n_layers, 4, t_copy);
        t_work = t_sfull = t_copy = 0;
      }
      const int nt = tile + n_pairs;
      if (nt < n_tiles) {
        if (et < NZV) zpref = load_z(a, nt * NPC + et / NZ, et % NZ);
        if (!(ok = input_layer(nt, it + 1))) break;
      }
      // output layer (slot 1): rank 0's TMEM lanes 0..2 hold the three outputs
      if (!(ok = wwait(acc_full(1), (acc_par >> 1) & 1u))) break;
      acc_par ^= 2u;
      if (tr) trace(a, it, nh, n_layers, 2);
      tc_fence_after();
      if (rank == 0 && q == 0) {
        const uint32_t tout = tmem + NMMA;  // accumulator slot 1
        float tl[TAIL];
#pragma unroll
        for (int c = 0; c < TAIL / 16; ++c) tmem_ld16_sum<C, 2>(tout + 16 * NPC + 16 * c, tl + 16 * c);
        tmem_wait_ld();
        const float bo = lane < NO ? a.bias[(size_t)nh * HP + lane] : 0.0f;
#pragma unroll
        for (int n = 0; n < NPC; ++n) {
          if ((n < HALF) != (half == 0)) continue;
          float t[16];
          tmem_ld16_sum<C, 2>(tout + 16 * n, t);
          tmem_wait_ld();
          const int node = node0 + n;
          if (lane < NO && node < a.n_nodes) {
            a.fD[(size_t)node * NO + lane] = tl[n] + bo;
            float* J = a.JD + (size_t)node * NO * NZ + lane * NZ;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) J[jj] = t[jj];
            J[16] = tl[NPC + n];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) arrive_cluster_relaxed(tf0 + 8u);
    }
    // tail: the last output layer's release of every block (its commit
    // reaches both CTAs)
    if (ok && it > 0)
      for (int j = 0; j < nblk && ok; ++j) ok = wwait(xfree(j), (uint32_t)(n_layers * it - 1) & 1u);
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

// kernel entry points of the pair variants (registered in mlp_tc.cu)
const void* mlp_tc2_fn(int npc, int stages) {
  if (npc == 7 && stages == 4) return (const void*)&mlp_tc2_kernel<7, 4>;
  if (npc == 6 && stages == 5) return (const void*)&mlp_tc2_kernel<6, 5>;
  if (npc == 7 && stages == 8) return (const void*)&mlp_tc2_kernel<7, 8>;
  if (npc == 4 && stages == 6) return (const void*)&mlp_tc2_kernel<4, 6>;
  return nullptr;
}

}  // namespace rtn

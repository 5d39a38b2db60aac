// One persistent launch for a batch of independent exchange problems (cells, grids and orbital
// counts may all differ).
//
// Work is a list of tasks; a task is one pass of one batch of pair couples of one problem (the
// forward plane pass, the x/Coulomb pass or the inverse-y accumulate pass) or the final energy
// sum of a problem, and consists of `items` independent items (planes, tiles).  The items of all
// tasks are numbered in task order; every block of the launch repeatedly takes the next item
// number from a global counter, runs that item and counts it done for its task.  The tasks of one
// problem form a chain (forward b -> x b -> accumulate b -> forward b+1 -> ... -> energy), so a
// task's items may start only when its predecessor's items are all done: the block that took the
// item waits for that, reading the predecessor's done counter, for at most `budget` clock cycles.
// The tasks of different problems are interleaved (level by level), so while one problem waits,
// the items of the others keep every SM busy.
//
// The wait cannot deadlock: items are taken in task order, so every item of a predecessor was
// taken before the waiting item, by a block that is running, and that block only ever waits on
// items taken before its own.  If a wait still runs out of budget (nothing completes the
// predecessor -- only the failure-detection test arranges that), the block sets kErrTimeout in
// the problem's error word and an abort flag, and every block returns at its next item or wait;
// the results of that call are then undefined and hfx_sync_status reports HFX_ERR_TIMEOUT.
#pragma once
#include <type_traits>

#include "hfx_ct.cuh"
#include "hfx_kernels.cuh"

namespace hfx {

enum BatchKind : int { kTaskFwd = 0, kTaskX = 1, kTaskAcc = 2, kTaskEnergy = 3, kTaskWiden = 4 };

constexpr int kWidenPerItem = 4096;  // elements of V_x phi per widening item

template <typename T>
struct BatchProblem {
  Geo g;
  const T* orb;                 // orbitals the passes read (the FP32 copy on the FP32 path)
  const int4* couples;          // staged pair couples
  cx<T>* W;                     // the problem's transform buffer (one batch at a time)
  double* epart;                // per-couple, per-y-plane energy partial sums
  T* V;                         // V_x phi accumulator (FP64, or the call's FP32 one)
  double* V64;                  // V_x phi (FP64) the FP32 accumulator is widened into
  long long n_v;                // elements of V_x phi
  double* ex;                   // E_x (FP64 scalar)
  const T* vtab;                // v(G) in storage order
  const cx<T>* tw1;
  const cx<T>* tw2;
  const cx<T>* tw3;
  const int* slot_couple_base;
  const int2* slot_blocks;
  const cx<T>* twct;            // per-stage twiddles of the compile-time passes (ct_n > 0)
  int* err;                     // the problem's context error word
  double vscale, escale;
  int n_orb, bsize, grp, phi_smem, cap_max, total_couples, accumulate, energy_only;
  int ct_n;                     // cubic FP32 edge with compile-time forward and x passes, else 0
};

// forward / x item of an FP32 problem through the compile-time passes of its edge; false when the
// problem has none (the runtime-geometry item runs instead)
// (tw_ok: the twiddle table of edge N is already in shared memory from this block's previous item)
template <typename T, int N>
__device__ __forceinline__ bool ct_item_n(const BatchProblem<T>& P, int kind, int a0, long long local,
                                          unsigned char* smem_raw, float (*redf)[32], int par, bool tw_ok) {
  if constexpr (std::is_same<T, float>::value) {
    if (P.ct_n != N) return false;
    constexpr StagePlan SP = ct::Plan<N>::p;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* tw = buf + N * (N + 1);
    if (!tw_ok)
      for (int i = threadIdx.x; i < SP.twtotal; i += blockDim.x) tw[i] = P.twct[i];
    if (kind == kTaskFwd)
      ct::fwd_yz_ct_item<float, N>(P.orb, P.g.N, P.couples, a0, P.W, buf, tw, (int)local);
    else
      ct::x_coulomb_ct_item<float, N>(P.couples, a0, P.W, P.vtab, P.epart, P.energy_only, buf, tw, redf, par,
                                      (int)local);
    return true;
  } else {
    return false;
  }
}

template <typename T>
__device__ __forceinline__ bool ct_item(const BatchProblem<T>& P, int kind, int a0, long long local,
                                        unsigned char* smem_raw, float (*redf)[32], int par, bool tw_ok) {
  return ct_item_n<T, 48>(P, kind, a0, local, smem_raw, redf, par, tw_ok) ||
         ct_item_n<T, 64>(P, kind, a0, local, smem_raw, redf, par, tw_ok) ||
         ct_item_n<T, 72>(P, kind, a0, local, smem_raw, redf, par, tw_ok) ||
         ct_item_n<T, 80>(P, kind, a0, local, smem_raw, redf, par, tw_ok) ||
         ct_item_n<T, 90>(P, kind, a0, local, smem_raw, redf, par, tw_ok) ||
         ct_item_n<T, 96>(P, kind, a0, local, smem_raw, redf, par, tw_ok);
}

struct BatchTask {
  long long first;  // number of this task's first item
  int items;
  int prob;
  int kind;
  int a0, a1;       // couple range [a0, a1) (forward, x) or slot range (accumulate)
  int cbase;        // first couple of the batch (its couple 0 in the transform buffer)
  int dep;          // predecessor task (-1: none)
  int extra;        // added to the predecessor's item count the wait expects (failure-detection test)
  int pad;
};

struct BatchQueue {
  unsigned long long next;  // next item number to hand out
  int abort;
  int pad;
  // followed by one done counter per task
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kThreadsBatch = 256;
// resident blocks per SM the persistent kernel is built for (registers: FP64 items need more)
template <typename T> struct BatchMinBlocks { static constexpr int value = sizeof(T) == 4 ? 3 : 1; };

template <typename T>
__global__ void __launch_bounds__(kThreadsBatch, BatchMinBlocks<T>::value)
k_batch_persistent(const BatchProblem<T>* __restrict__ probs, const BatchTask* __restrict__ tasks, int ntasks,
                   long long total_items, BatchQueue* queue, long long budget) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  __shared__ int s_task;
  __shared__ double red[32];
  __shared__ float redf[2][32];  // warp partials of the compile-time x items, alternating
  int par = 0;
  int* done = reinterpret_cast<int*>(queue + 1);
  int cur = 0;         // thread 0: the task of this block's previous item (items only increase)
  int ct_loaded = 0;   // edge whose compile-time twiddle table this block's shared memory holds
  for (;;) {
    if (threadIdx.x == 0) {
      int task = -1;
      long long item = 0;
      if (!*(volatile int*)&queue->abort) {
        item = (long long)atomicAdd(&queue->next, 1ull);
        if (item < total_items) {
          // the last task whose first item <= item, scanning on from the previous one
          while (cur + 1 < ntasks && tasks[cur + 1].first <= item) ++cur;
          task = cur;
          const BatchTask tk = tasks[task];
          if (tk.dep >= 0) {
            const int target = tasks[tk.dep].items + tk.extra;
            const long long t0 = clock64();
            while (ld_acquire_gpu(done + tk.dep) < target) {
              if (*(volatile int*)&queue->abort) { task = -1; break; }
              if (clock64() - t0 > budget) {
                atomicOr(probs[tk.prob].err, kErrTimeout);
                atomicExch(&queue->abort, 1);
                task = -1;
                break;
              }
              __nanosleep(256);
            }
          }
        }
      }
      s_item = item;
      s_task = task;
    }
    __syncthreads();
    const int task = s_task;
    if (task < 0) return;
    const BatchTask tk = tasks[task];
    const BatchProblem<T>& P = probs[tk.prob];
    const long long local = s_item - tk.first;
    const Geo& g = P.g;
    if ((tk.kind == kTaskFwd || tk.kind == kTaskX) && P.ct_n > 0 &&
        ct_item(P, tk.kind, tk.a0, local, smem_raw, redf, par, ct_loaded == P.ct_n)) {
      if (tk.kind == kTaskX) par ^= 1;
      ct_loaded = P.ct_n;
    } else if (tk.kind == kTaskFwd) {
      ct_loaded = 0;  // the items below reuse the shared memory that held a twiddle table
      C* buf = reinterpret_cast<C*>(smem_raw);
      C* tw2 = buf + g.n2 * g.S;
      C* tw3 = tw2 + g.n2;
      for (int i = threadIdx.x; i < g.n2; i += blockDim.x) tw2[i] = P.tw2[i];
      for (int i = threadIdx.x; i < g.n3; i += blockDim.x) tw3[i] = P.tw3[i];
      fwd_yz_item(g, P.orb, P.couples, tk.a0, P.W, tw2, tw3, buf, local);
    } else if (tk.kind == kTaskX) {
      ct_loaded = 0;
      C* buf = reinterpret_cast<C*>(smem_raw);
      C* tw1 = buf + g.n1 * g.S;
      C* tw3 = tw1 + g.n1;
      for (int i = threadIdx.x; i < g.n1; i += blockDim.x) tw1[i] = P.tw1[i];
      for (int i = threadIdx.x; i < g.n3; i += blockDim.x) tw3[i] = P.tw3[i];
      x_coulomb_item(g, P.couples, tk.a0, P.W, P.vtab, tw1, tw3, P.epart, P.energy_only != 0, buf, red, local);
    } else if (tk.kind == kTaskAcc) {
      ct_loaded = 0;
      constexpr int ZC = ZChunk<T>::value;
      const int nzc = (g.n3 + ZC - 1) / ZC;
      const int zi = int(local % nzc);
      const long long rest = local / nzc;
      const int x = int(rest % g.n1);
      const int slot = tk.a0 + int(rest / g.n1);
      acc_generic_item(g, P.orb, P.couples, slot, P.slot_couple_base, P.slot_blocks, P.bsize, P.n_orb, tk.cbase, P.W,
                       P.tw2, P.V, P.vscale, P.grp, P.phi_smem, P.cap_max, smem_raw, zi, x);
    } else if (tk.kind == kTaskWiden) {
      // V_x phi (FP64) = (accumulate ? V_x phi : 0) + the FP32 accumulator, widened exactly
      const long long e0 = local * kWidenPerItem;
      for (int i = threadIdx.x; i < kWidenPerItem / 4; i += blockDim.x) {
        const long long e = e0 + 4LL * i;
        if (e + 4 > P.n_v) break;
        const float4 a = __ldcg(reinterpret_cast<const float4*>(P.V) + e / 4);
        double2* d = reinterpret_cast<double2*>(P.V64 + e);
        double2 lo = make_double2(ct::widen_exact(a.x), ct::widen_exact(a.y));
        double2 hi = make_double2(ct::widen_exact(a.z), ct::widen_exact(a.w));
        if (P.accumulate) {
          const double2 o0 = d[0], o1 = d[1];
          lo.x += o0.x; lo.y += o0.y; hi.x += o1.x; hi.y += o1.y;
        }
        d[0] = lo;
        d[1] = hi;
      }
    } else {  // energy: E_x = scale * sum_g w_g sum_y epart[g][y], in a fixed order
      ct_loaded = 0;  // (block_sum below uses only static shared memory; kept simple)
      double sacc = 0.0;
      for (int c = threadIdx.x; c < P.total_couples; c += blockDim.x) {
        const int4 cp = P.couples[c];
        if (couple_empty(cp)) continue;
        const bool diag = cp.x >= 0 ? cp.x == cp.y : cp.z == cp.w;
        double t = 0.0;
        for (int y = 0; y < g.n2; ++y) t += __ldcg(P.epart + (long long)c * g.n2 + y);
        sacc += (diag ? 1.0 : 2.0) * t;
      }
      const double tot = block_sum(sacc, red);
      if (threadIdx.x == 0) P.ex[0] = (P.accumulate ? P.ex[0] : 0.0) + P.escale * tot;
    }
    __syncthreads();  // the item's writes are done (and its shared memory is free)
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + task, 1);
    }
  }
}

}  // namespace hfx

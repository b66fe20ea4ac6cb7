// nb_symsched.cuh -- the work schedule of the half-pair (symmetric) kernels
// and their in-place, ordered accumulation.
//
// Ions are grouped in nbk blocks.  A work item is a block pair (P, Q), P <= Q:
// P < Q evaluates every pair between the two blocks once and yields a sum
// for each ion of both; P == Q yields the block's internal sums.  Every
// block takes part in exactly one item per round, so within a round the
// items touch disjoint blocks (a round-robin tournament, "circle method"):
//  - nbk odd: nbk rounds of (nbk + 1) / 2 items.  A dummy block nbk joins the
//    rotation; block r meets it in round r and does its diagonal item then.
//    Round r pairs (r + k) mod nbk with (r - k) mod nbk, k = 1 .. (nbk-1)/2.
//  - nbk even: round 0 holds the nbk diagonal items; rounds 1 .. nbk-1 pair
//    block nbk-1 with block r-1 and (r-1 + k) mod (nbk-1) with
//    (r-1 - k) mod (nbk-1), k = 1 .. nbk/2 - 1.
// Either way there are nbk (nbk + 1) / 2 items, numbered round by round.
//
// Accumulation.  The item of round r adds its sums into the caller's output
// acc[c][i] (c = x, y, z) of both blocks -- round 0 stores them -- after the
// items of round r - 1 that touched the same blocks have added theirs.  So
// every ion's sum is formed in round order, whatever order the items run
// in, and the result is bitwise reproducible with no partial-sum buffer:
// the output itself is the only accumulator, 3 n doubles, which L2 holds.
// (sym_output below also offers the per-partner-block partials for small
// schedules.)
//
// Ordering and progress.  A block of the grid draws its item number from a
// counter (atomicAdd) when it starts, so item t runs only after every item
// below t has been drawn by a block that is already resident.  An item waits
// only for lower-numbered items (the previous round), so the lowest
// unfinished item never waits and the grid always progresses.  The wait is a
// bounded spin on the per-block round counters with acquire loads; the
// writer's threads meet at a barrier, then its thread 0 fences and
// publishes with a release store.  A wait that runs out
// sets ERR_TIMEOUT in the stream's error word and skips its adds (the
// result is then wrong and flagged; the kernel still ends).
//
// sync[0] is the item counter and sync[1 + b] the number of rounds
// committed for block b; both are zeroed before every launch.
#pragma once

#include "nb_common.cuh"

namespace nb {

// Spins of about 0.1-0.3 us each before a wait gives up (well over a second;
// a wait normally lasts a few microseconds at most).
constexpr int SYM_SPIN_LIMIT = 1 << 23;

// Number of ints of sync state for nbk blocks.
__host__ __device__ constexpr int64_t sym_sync_ints(int64_t nbk) { return nbk + 1; }

struct SymItem {
  int P, Q, round;
};

// Item t of the schedule above (0 <= t < nbk (nbk + 1) / 2).  Also compiled
// for the host, where nb_sym_schedule lists the schedule for tests.
__host__ __device__ __forceinline__ SymItem sym_item(int t, int nbk) {
  SymItem it;
  if (nbk & 1) {
    const int per = (nbk + 1) >> 1;
    const int r = t / per, k = t - r * per;
    it.round = r;
    if (k == 0) {
      it.P = it.Q = r;
    } else {
      const int a = (r + k) % nbk, b = (r - k + nbk) % nbk;
      it.P = a < b ? a : b;
      it.Q = a < b ? b : a;
    }
  } else if (t < nbk) {
    it.P = it.Q = t;
    it.round = 0;
  } else {
    const int m = nbk - 1, per = nbk >> 1, u = t - nbk;
    const int r = u / per, k = u - r * per;
    it.round = r + 1;
    if (k == 0) {
      it.P = r;
      it.Q = m;
    } else {
      const int a = (r + k) % m, b = (r - k + m) % m;
      it.P = a < b ? a : b;
      it.Q = a < b ? b : a;
    }
  }
  return it;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until block b has committed `round` rounds.  It also gives
// up at once when another block's wait has already run out (the error word
// has ERR_TIMEOUT), so a failing launch ends after one spin limit, not one
// per item.
__device__ __forceinline__ bool sym_wait(const int *sync, int b, int round, const unsigned *err) {
  for (int it = 0; it < SYM_SPIN_LIMIT; ++it) {
    if (ld_acquire(sync + 1 + b) >= round) return true;
    if ((it & 255) == 255 && (*(const volatile unsigned *)err & ERR_TIMEOUT)) return false;
    __nanosleep(64);
  }
  return false;
}

// Item number of this block (thread 0 draws, the block shares it).
__device__ __forceinline__ int sym_draw(int *sync) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = atomicAdd(sync, 1);
  __syncthreads();
  return s_t;
}

// Adds the item's sums into acc after the previous round's items of the same
// blocks: sumP(c, i) for the np ions of block P at p0, and (P != Q) sumQ(c, i)
// for the nq ions of block Q at q0.  Called by every thread of the block.
template <int NT, class FP, class FQ>
__device__ __forceinline__ void sym_commit(const SymItem &it, int64_t n, int64_t p0, int np, int64_t q0, int nq,
                                           double *acc, int *sync, unsigned *err, FP sumP, FQ sumQ) {
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  if (tid == 0) {
    bool ok = true;
    if (it.round > 0)
      ok = sym_wait(sync, it.P, it.round, err) && (it.P == it.Q || sym_wait(sync, it.Q, it.round, err));
    if (!ok) atomicOr(err, ERR_TIMEOUT);
    s_ok = ok;
  }
  __syncthreads();
  if (s_ok) {
    const bool first = it.round == 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double *a = acc + (int64_t)c * n;
      for (int i = tid; i < np; i += NT) {
        const double v = sumP(c, i);
        __stcg(a + p0 + i, first ? v : __ldcg(a + p0 + i) + v);
      }
      if (it.P != it.Q)
        for (int i = tid; i < nq; i += NT) {
          const double v = sumQ(c, i);
          __stcg(a + q0 + i, first ? v : __ldcg(a + q0 + i) + v);
        }
    }
  }
  __syncthreads();  // every thread's adds happen before thread 0's release
  if (tid == 0) {
    __threadfence();
    st_release(sync + 1 + it.P, it.round + 1);
    if (it.P != it.Q) st_release(sync + 1 + it.Q, it.round + 1);
  }
}

// The item's output in either of the two modes of the half-pair kernels:
//  - inplace: sym_commit, the round-ordered adds into acc ([3][n], no
//    partial buffer); used when there are many items per resident block, so
//    the rounds' commits overlap the arithmetic of later rounds;
//  - partials: one slot per partner block, acc[(X * 3 + c) * n + i] for the
//    sum over block X, which the epilogue adds in block order; used when the
//    items fit in a few waves, where the chain of nbk commits would follow
//    the arithmetic instead of overlapping it.
template <int NT, class FP, class FQ>
__device__ __forceinline__ void sym_output(bool inplace, const SymItem &it, int64_t n, int64_t p0, int np,
                                           int64_t q0, int nq, double *acc, int *sync, unsigned *err, FP sumP,
                                           FQ sumQ) {
  if (inplace) {
    sym_commit<NT>(it, n, p0, np, q0, nq, acc, sync, err, sumP, sumQ);
    return;
  }
  const int tid = threadIdx.x;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    for (int i = tid; i < np; i += NT) acc[((int64_t)it.Q * 3 + c) * n + p0 + i] = sumP(c, i);
    if (it.P != it.Q)
      for (int i = tid; i < nq; i += NT) acc[((int64_t)it.P * 3 + c) * n + q0 + i] = sumQ(c, i);
  }
}

// The item a block works on: drawn from the counter in the in-place mode
// (so that waits point only at running items), blockIdx.x otherwise.
__device__ __forceinline__ SymItem sym_block_item(bool inplace, int *sync, int nbk) {
  return sym_item(inplace ? sym_draw(sync) : (int)blockIdx.x, nbk);
}

}  // namespace nb

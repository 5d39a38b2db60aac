// Pair-block schedule of one exchange evaluation (host code, no device work): which orbital-block
// pairs exist, the rounds in which no two of them share a block, the batches that the transform
// budget cuts the rounds into, the couple capacity of every block pair in the canonical layout,
// and which accumulation pass takes each block pair.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <vector>

namespace hfx {

// ------------------------------------------------------------------------------------
// pair-block schedule for n_orb orbitals in blocks of `b`: block pairs (I <= J) are arranged
// in rounds in which no two block pairs share a block (circle method), so every V_x phi tile
// of a round has one writer; rounds are cut into batches by the transform budget.
// ------------------------------------------------------------------------------------
struct Schedule {
  int n_orb = 0, b = 0, nb = 0, nslots = 0, nbatches = 0;
  std::vector<int2> slot_blocks;        // slot -> (I, J)
  std::vector<int> slot_of_bp;          // I*nb + J (I <= J) -> slot
  std::vector<int> slot_cap;            // couples a slot holds (canonical layout, holes allowed)
  std::vector<int> slot_couple_base;    // [nslots + 1], prefix of slot_cap
  std::vector<int> batch_slot_begin;    // [nbatches + 1]
  // per batch: slots taken by the dense accumulation kernel and by the generic one
  std::vector<int> dense_slots, generic_slots, diag_slots;  // concatenated over batches
  std::vector<int> dense_begin, generic_begin, diag_begin;  // [nbatches + 1] offsets into the lists
  long long max_batch_couples = 0, max_total_couples = 0;
  // device copies
  int2* d_slot_blocks = nullptr;
  int* d_slot_of_bp = nullptr;
  int* d_slot_couple_base = nullptr;
  int* d_dense_slots = nullptr;
  int* d_generic_slots = nullptr;
  int* d_diag_slots = nullptr;
};

static int block_size_of(int bi, int b, int n_orb) { return std::min(b, n_orb - bi * b); }

// couples of a slot in the canonical layout: I != J: all sI sJ pairs, couple t/2 of
// t = (i - I0) sJ + (j - J0); I == J: the sI (sI-1)/2 pairs i < j first, then the sI diagonal ones.
static int slot_capacity(int si, int sj, bool diag) {
  if (!diag) return (si * sj + 1) / 2;
  return (si * (si - 1) / 2 + 1) / 2 + (si + 1) / 2;
}

static void build_schedule(Schedule& S, int n_orb, int b, size_t transform_budget, size_t bytes_per_couple,
                           bool dense_ok, bool diag_ok) {
  S.n_orb = n_orb;
  S.b = b;
  S.nb = (n_orb + b - 1) / b;
  const int nb = S.nb;
  std::vector<std::vector<int2>> rounds;
  if (nb == 1) {
    rounds.push_back({make_int2(0, 0)});
  } else {
    const int M = (nb % 2 == 0) ? nb : nb + 1;  // with a dummy block when odd
    const int fixed = M - 1;
    for (int r = 0; r < M - 1; ++r) {
      std::vector<int2> rd;
      auto add = [&](int a, int c) {
        if (a >= nb && c >= nb) return;
        if (a >= nb) { rd.push_back(make_int2(c, c)); return; }   // partner is the dummy: diagonal
        if (c >= nb) { rd.push_back(make_int2(a, a)); return; }
        rd.push_back(make_int2(std::min(a, c), std::max(a, c)));
      };
      add(r, fixed);
      for (int k = 1; k < M / 2; ++k) add((r + k) % (M - 1), (r - k + (M - 1)) % (M - 1));
      rounds.push_back(rd);
    }
    if (nb % 2 == 0) {
      std::vector<int2> rd;
      for (int i = 0; i < nb; ++i) rd.push_back(make_int2(i, i));
      rounds.push_back(rd);
    }
  }
  S.slot_blocks.clear();
  S.slot_cap.clear();
  S.batch_slot_begin.clear();
  S.slot_of_bp.assign((size_t)nb * nb, -1);
  S.max_batch_couples = 0;
  S.max_total_couples = 0;
  const long long budget_couples = std::max<long long>(1, (long long)(transform_budget / bytes_per_couple));
  for (auto& rd : rounds) {
    long long in_batch = 0;
    bool open = false;
    for (auto bp : rd) {
      const int si = block_size_of(bp.x, b, n_orb), sj = block_size_of(bp.y, b, n_orb);
      const int cap = slot_capacity(si, sj, bp.x == bp.y);
      if (!open || in_batch + cap > budget_couples) {
        if (open) S.max_batch_couples = std::max(S.max_batch_couples, in_batch);
        S.batch_slot_begin.push_back((int)S.slot_blocks.size());
        in_batch = 0;
        open = true;
      }
      S.slot_of_bp[(size_t)bp.x * nb + bp.y] = (int)S.slot_blocks.size();
      S.slot_blocks.push_back(bp);
      S.slot_cap.push_back(cap);
      in_batch += cap;
      S.max_total_couples += cap;
    }
    if (open) S.max_batch_couples = std::max(S.max_batch_couples, in_batch);
  }
  S.nslots = (int)S.slot_blocks.size();
  S.nbatches = (int)S.batch_slot_begin.size();
  S.batch_slot_begin.push_back(S.nslots);
  S.slot_couple_base.assign(S.nslots + 1, 0);
  for (int k = 0; k < S.nslots; ++k) S.slot_couple_base[k + 1] = S.slot_couple_base[k] + S.slot_cap[k];
  S.dense_slots.clear();
  S.generic_slots.clear();
  S.diag_slots.clear();
  S.dense_begin.assign(1, 0);
  S.generic_begin.assign(1, 0);
  S.diag_begin.assign(1, 0);
  for (int bt = 0; bt < S.nbatches; ++bt) {
    for (int k = S.batch_slot_begin[bt]; k < S.batch_slot_begin[bt + 1]; ++k) {
      const int2 bp = S.slot_blocks[k];
      const bool full = block_size_of(bp.x, b, n_orb) == b && block_size_of(bp.y, b, n_orb) == b;
      if (dense_ok && bp.x != bp.y && full) S.dense_slots.push_back(k);
      else if (diag_ok && bp.x == bp.y && full) S.diag_slots.push_back(k);
      else S.generic_slots.push_back(k);
    }
    S.dense_begin.push_back((int)S.dense_slots.size());
    S.generic_begin.push_back((int)S.generic_slots.size());
    S.diag_begin.push_back((int)S.diag_slots.size());
  }
}

}  // namespace hfx

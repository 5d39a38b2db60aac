// Prints, as one JSON object, the pair-block schedule that libhfx builds for
//   n_orb  block  transform_budget_bytes  bytes_per_couple  dense_ok  diag_ok
// (the library's own build_schedule, host code only), for tests/test_schedule_host.py.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2309_00651_gb300/csrc/hfx_schedule.h"

static void ints(const char* name, const std::vector<int>& v, bool last = false) {
  std::printf("\"%s\": [", name);
  for (size_t i = 0; i < v.size(); ++i) std::printf("%s%d", i ? ", " : "", v[i]);
  std::printf("]%s\n", last ? "" : ",");
}

int main(int argc, char** argv) {
  if (argc != 7) {
    std::fprintf(stderr, "usage: %s n_orb block budget_bytes bytes_per_couple dense_ok diag_ok\n", argv[0]);
    return 2;
  }
  hfx::Schedule S;
  hfx::build_schedule(S, std::atoi(argv[1]), std::atoi(argv[2]), (size_t)std::strtoull(argv[3], nullptr, 10),
                      (size_t)std::strtoull(argv[4], nullptr, 10), std::atoi(argv[5]) != 0, std::atoi(argv[6]) != 0);
  std::printf("{\"n_orb\": %d, \"b\": %d, \"nb\": %d, \"nslots\": %d, \"nbatches\": %d,\n", S.n_orb, S.b, S.nb,
              S.nslots, S.nbatches);
  std::printf("\"max_batch_couples\": %lld, \"max_total_couples\": %lld,\n", S.max_batch_couples,
              S.max_total_couples);
  std::printf("\"slot_blocks\": [");
  for (size_t i = 0; i < S.slot_blocks.size(); ++i)
    std::printf("%s[%d, %d]", i ? ", " : "", S.slot_blocks[i].x, S.slot_blocks[i].y);
  std::printf("],\n");
  ints("slot_of_bp", S.slot_of_bp);
  ints("slot_cap", S.slot_cap);
  ints("slot_couple_base", S.slot_couple_base);
  ints("batch_slot_begin", S.batch_slot_begin);
  ints("dense_slots", S.dense_slots);
  ints("dense_begin", S.dense_begin);
  ints("generic_slots", S.generic_slots);
  ints("generic_begin", S.generic_begin);
  ints("diag_slots", S.diag_slots);
  ints("diag_begin", S.diag_begin, true);
  std::printf("}\n");
  return 0;
}

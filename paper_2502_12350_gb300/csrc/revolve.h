// Checkpoint schedule (internal to libmamute).
#pragma once

#include <vector>

namespace mamute {

enum RevKind { REV_ADVANCE = 0, REV_STORE = 1, REV_RESTORE = 2, REV_REVERSE = 3 };

struct RevAction {
  int kind, a, b;  // ADVANCE a->b; STORE slot a (state b); RESTORE slot a (state b); REVERSE step a
};

// Minimum forward steps to reverse l steps from a held state with s free slots.
long long revolve_cost(long long l, int s);

// Plan for nt steps from the zero state with n_slots slots.  n_forward counts
// every forward step, including the one that produces the last data sample.
int revolve_plan(int nt, int n_slots, std::vector<RevAction>& actions, long long& n_forward);

}  // namespace mamute

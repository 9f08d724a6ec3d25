// Binomial checkpointing plan (Sec. 2.1: optimal checkpointing of the
// forward wavefield after Griewank and Walther's revolve; Table 4 check_mem
// sizes the slot count).
//
// Reversing l steps from a held, restorable state x_a with s free slots:
//   l == 1: reverse step a;
//   s == 0: for each step from last to first, restore x_a, advance to it and
//           reverse it;
//   else:   advance j steps, store x_{a+j} in a free slot, reverse the right
//           part with s-1 slots, restore x_a, reverse the left part with s
//           slots, with j minimising j + C(l-j, s-1) + C(j, s).
// C(l, s) is the closed-form minimum t l - beta(s+2, t-1), t the least integer
// with beta(s+1, t) >= l, beta(a, t) = (a+t)! / (a! t!).
#include "revolve.h"

#include <algorithm>
#include <cmath>

namespace mamute {

namespace {

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return std::floor(r + 0.5);
}

long long closed_cost(long long l, int s) {
  if (l <= 1) return 0;
  if (s == 0) return l * (l - 1) / 2;
  int t = 0;
  while (binom(s + 1 + t, t) < (double)l) ++t;
  return (long long)t * l - (long long)binom(s + 2 + t - 1, t - 1);
}

struct Planner {
  int nt, S;
  std::vector<long long> table;  // C(l, s) for l <= nt, s <= S
  std::vector<RevAction>* out;
  long long nfwd = 0;

  long long C(long long l, int s) const {
    if (l <= 1) return 0;
    return table[(size_t)l * (S + 1) + s];
  }

  void emit(int k, int a, int b) { out->push_back(RevAction{k, a, b}); }

  // Current state is x_a, held in slot `held` (-1: the zero initial state).
  void rev(int a, int l, std::vector<int>& free_slots, int held, bool at_a) {
    if (l == 1) {
      if (!at_a) emit(REV_RESTORE, held, a);
      emit(REV_REVERSE, a, 0);
      return;
    }
    const int s = (int)free_slots.size();
    if (s == 0) {
      for (int i = l - 1; i >= 0; --i) {
        if (!at_a) emit(REV_RESTORE, held, a);
        if (i > 0) {
          emit(REV_ADVANCE, a, a + i);
          nfwd += i;
        }
        emit(REV_REVERSE, a + i, 0);
        at_a = false;
      }
      return;
    }
    int best = 1;
    long long bc = -1;
    for (int j = 1; j < l; ++j) {
      const long long c = j + C(l - j, s - 1) + C(j, s);
      if (bc < 0 || c < bc) {
        bc = c;
        best = j;
      }
    }
    if (!at_a) emit(REV_RESTORE, held, a);
    emit(REV_ADVANCE, a, a + best);
    nfwd += best;
    const int slot = free_slots.back();
    free_slots.pop_back();
    emit(REV_STORE, slot, a + best);
    rev(a + best, l - best, free_slots, slot, true);
    free_slots.push_back(slot);
    rev(a, best, free_slots, held, false);
  }
};

}  // namespace

long long revolve_cost(long long l, int s) { return closed_cost(l, s); }

int revolve_plan(int nt, int n_slots, std::vector<RevAction>& actions, long long& n_forward) {
  actions.clear();
  n_forward = 0;
  if (nt < 1 || n_slots < 0) return -1;
  Planner P;
  P.nt = nt;
  P.S = std::min(n_slots, nt);
  P.table.assign((size_t)(nt + 1) * (P.S + 1), 0);
  for (int l = 0; l <= nt; ++l)
    for (int s = 0; s <= P.S; ++s) P.table[(size_t)l * (P.S + 1) + s] = closed_cost(l, s);
  P.out = &actions;
  std::vector<int> free_slots;
  for (int k = P.S - 1; k >= 0; --k) free_slots.push_back(k);
  P.rev(0, nt, free_slots, -1, true);
  // One more forward step from the last state produces the final data sample.
  n_forward = P.nfwd + 1;
  return 0;
}

}  // namespace mamute

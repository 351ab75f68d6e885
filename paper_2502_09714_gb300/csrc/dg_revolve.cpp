// Binomial checkpointing of the step history for the discrete adjoint
// (Griewank's revolve): reversing n steps with s snapshot slots besides the
// retained initial state.  The plan is the recursion
//     reverse(l, r, s): advance l -> l + m, store l + m, reverse(l + m, r, s - 1),
//                       restore l, reverse(l, l + m, s)
// with a split m that minimises the forward steps, whose optimum has the
// closed form  T(n, s) = t n - C(s + 1 + t, t - 1),  t the least integer with
// C(s + 1 + t, t) >= n  (T(n, 0) = n (n - 1) / 2, T(1, s) = 0).  Each level of the
// recursion lowers s or t, so its depth stays below s + t.  The adjoint of
// step j needs the state Q^j in hand; it recomputes its own predictor.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "dg.h"
#include "dg_revolve.h"

namespace dg {

namespace {

// C(a + t, t), saturated at 2^62
int64_t beta(int64_t a, int64_t t) {
  if (t < 0) return 0;
  long double c = 1.0L;
  for (int64_t j = 1; j <= t; ++j) {
    c = c * static_cast<long double>(a + j) / static_cast<long double>(j);
    if (c > 4.6e18L) return int64_t(1) << 62;
  }
  return static_cast<int64_t>(c + 0.5L);
}

struct Planner {
  std::vector<RevolveAction>* out;
  std::vector<int> free_slots;

  void emit(int kind, int64_t a, int64_t b) { out->push_back(RevolveAction{kind, a, b}); }

  // An optimal first split: with t the repetition number of (n, s), C(s + t, t) < n at t - 1,
  // m = max(C(s + t - 1, t - 2), n - C(s + t, t)) leaves a right part of n - m steps that s - 1
  // slots reverse with t repetitions and a left part that s slots reverse with t - 1.
  static int64_t split(int64_t n, int s) {
    int64_t t = 0;
    while (beta(s + 1, t) < n) ++t;
    const int64_t m = std::max(beta(s + 1, t - 2), n - beta(s, t));
    return std::min(std::max<int64_t>(m, 1), n - 1);
  }

  void reverse(int64_t l, int64_t r, int s, int slot_l) {
    const int64_t n = r - l;
    if (n <= 0) return;
    if (n == 1) {
      emit(kRestore, slot_l, l);
      emit(kAdjoint, l, 0);
      return;
    }
    if (s == 0) {
      for (int64_t j = r - 1; j >= l; --j) {
        emit(kRestore, slot_l, l);
        if (j > l) emit(kAdvance, l, j);
        emit(kAdjoint, j, 0);
      }
      return;
    }
    const int64_t m = split(n, s);
    emit(kRestore, slot_l, l);
    emit(kAdvance, l, l + m);
    const int slot = free_slots.back();
    free_slots.pop_back();
    emit(kStore, slot, l + m);
    reverse(l + m, r, s - 1, slot);
    free_slots.push_back(slot);
    reverse(l, l + m, s, slot_l);
  }
};

}  // namespace

int64_t revolve_cost(int64_t n, int s) {
  if (n <= 1) return 0;
  if (s <= 0) return n * (n - 1) / 2;
  int64_t t = 0;
  while (beta(s + 1, t) < n) ++t;
  return t * n - beta(s + 2, t - 1);
}

std::vector<RevolveAction> revolve_plan(int64_t n, int snapshots, int64_t* forward_steps) {
  std::vector<RevolveAction> out;
  Planner p{&out, {}};
  const int s = std::max(0, snapshots - 1);
  for (int k = s; k >= 1; --k) p.free_slots.push_back(k);
  p.reverse(0, n, s, 0);
  int64_t fw = 0;
  for (const RevolveAction& a : out)
    if (a.kind == kAdvance) fw += a.b - a.a;
  if (forward_steps) *forward_steps = fw;
  return out;
}

}  // namespace dg

extern "C" dg_status dg_revolve_plan(int64_t n_steps, int snapshots, int64_t* forward_steps, int64_t* actions,
                                     int64_t cap, int64_t* n_actions) {
  if (n_steps < 1 || n_steps > (int64_t(1) << 20) || snapshots < 1 || snapshots > 4096) return DG_E_ARG;
  if (dg::revolve_cost(n_steps, snapshots - 1) > dg::kMaxRevolveSteps) return DG_E_ARG;
  int64_t fw = 0;
  const std::vector<dg::RevolveAction> plan = dg::revolve_plan(n_steps, snapshots, &fw);
  if (forward_steps) *forward_steps = fw;
  if (n_actions) *n_actions = static_cast<int64_t>(plan.size());
  if (actions) {
    const int64_t n = std::min<int64_t>(cap, static_cast<int64_t>(plan.size()));
    for (int64_t i = 0; i < n; ++i) {
      actions[3 * i + 0] = plan[i].kind;
      actions[3 * i + 1] = plan[i].a;
      actions[3 * i + 2] = plan[i].b;
    }
  }
  return DG_OK;
}

extern "C" int64_t dg_revolve_cost(int64_t n_steps, int snapshots) {
  if (n_steps < 1 || snapshots < 1) return -1;
  return dg::revolve_cost(n_steps, snapshots - 1);
}

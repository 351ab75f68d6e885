// Binomial checkpointing plan of the discrete adjoint (dg_revolve.cpp).
// Internal to the library.
#pragma once

#include <cstdint>
#include <vector>

namespace dg {

enum : int {
  kAdvance = 0,   // step the current state from step a to step b
  kStore = 1,     // copy the current state (step b) into snapshot slot a
  kRestore = 2,   // make snapshot slot a (holding step b) the current state
  kAdjoint = 3,   // adjoint of step a (the current state is step a)
};
struct RevolveAction {
  int kind;
  int64_t a, b;
};

// Least number of forward steps that reverse n steps with s free slots
// besides the retained initial state.
int64_t revolve_cost(int64_t n, int s);
// The plan for n steps and `snapshots` state slots in all (slot 0 holds the
// initial state); *forward_steps receives the steps it advances.
std::vector<RevolveAction> revolve_plan(int64_t n, int snapshots, int64_t* forward_steps);

// Plans whose forward steps exceed this are refused.
constexpr int64_t kMaxRevolveSteps = int64_t(1) << 27;

}  // namespace dg

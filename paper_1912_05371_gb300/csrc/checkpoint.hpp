// Checkpoint schedules of the adjoint's reverse sweep (host only).
//
// The adjoint of n steps U_{k+1} = Phi_k(U_k) takes the steps' adjoints in the order n-1, ..., 0,
// each from its own state.  A schedule is a list of actions on a current state and numbered
// snapshots (device copies of a state):
//   STORE j     copy the current state into snapshot j
//   RESTORE j   make snapshot j the current state
//   ADVANCE k   the plain step k -> k+1 (the current state is U_k)
//   TURN k      step k with its adjoint, from U_k; the current state is used up
// Snapshot 0 receives U_0 as the first action and is never written again, so U_0 can always be
// put back.  A state is first reached in the order U_1, ..., U_n (U_n by TURN n-1), which is
// when the objective's terms are summed.
//
// equidistant(n, c): U_k is kept for every multiple k of c; in the backward sweep each segment
// of c steps is recomputed from its checkpoint with its states stored, then reversed (the last
// segment's states are stored on the first pass).  ceil(n/c) + max(c - 2, 0) snapshots.
//
// binomial(n, S): binomial checkpointing (Griewank 1992; Griewank and Walther, revolve, 2000)
// with S snapshots: to reverse steps a..b-1 from U_a with F further free snapshots, advance to
// some U_m, keep it, reverse m..b-1 with F-1 free, restore U_a and reverse a..m-1 with F free
// (no free snapshot: advance from U_a to each U_k in turn).  The split m minimises
// m + T(b-m, F) + T(m-a, F+1), T(n, S) the fewest advances, r n - C(S+r, r-1) with r the least
// integer with C(S+r, S) >= n; T is convex in n (its increments are r), so the smallest
// minimiser is found by bisection on the increments.  The result is that minimum.
#pragma once

#include <cstdint>
#include <vector>

namespace acm {
namespace ckpt {

enum Op : int8_t { STORE = 0, RESTORE = 1, ADVANCE = 2, TURN = 3 };

struct Action {
  int8_t op;
  int32_t arg;
};

struct Schedule {
  std::vector<Action> act;
  int32_t slots = 0;      // snapshots used (largest index + 1)
  int64_t advances = 0;   // plain forward steps (TURNs not counted)
};

constexpr int32_t kMaxSteps = 1 << 20;
// A schedule holds one action per recomputed step; longer ones are refused (few snapshots for
// very many steps: 2^20 steps with 2 snapshots would need about 1.5e9).
constexpr int64_t kMaxAdvances = int64_t(1) << 26;

// Fewest advances that reverse n steps with S snapshots (U_0's included).
inline int64_t binomial_advances(int64_t n, int64_t S) {
  if (n <= 1) return 0;
  if (S <= 1) return n * (n - 1) / 2;
  int64_t r = 0, beta = 1;                 // beta = C(S + r, S)
  while (beta < n) {
    ++r;
    beta = beta * (S + r) / r;             // exact: C(S+r, S) = C(S+r-1, S) (S+r) / r
  }
  return r * n - beta * r / (S + 1);       // C(S+r, r-1) = C(S+r, r) r / (S+1)
}

// Snapshots a policy needs: policy > 0 is equidistant every `policy` steps, policy < 0 binomial
// with -policy snapshots.  0 for an invalid policy or step count.
inline int64_t snapshots_needed(int64_t n, int64_t policy) {
  if (n < 1 || n > kMaxSteps || policy == 0) return 0;
  if (policy > 0) {
    const int64_t c = policy < n ? policy : n;
    const int64_t nck = (n - 1) / c + 1;
    return nck + (c > 2 ? c - 2 : 0);
  }
  const int64_t S = -policy < n ? -policy : n;
  return binomial_advances(n, S) > kMaxAdvances ? 0 : S;
}

inline void push(Schedule& s, Op op, int64_t arg) {
  s.act.push_back(Action{(int8_t)op, (int32_t)arg});
  if ((op == STORE || op == RESTORE) && arg + 1 > s.slots) s.slots = (int32_t)(arg + 1);
  if (op == ADVANCE) ++s.advances;
}

inline bool equidistant(int64_t n, int64_t policy, Schedule* out) {
  if (n < 1 || n > kMaxSteps || policy < 1) return false;
  Schedule s;
  const int64_t c = policy < n ? policy : n;
  const int64_t nck = (n - 1) / c + 1;
  const int64_t a_last = (nck - 1) * c;
  // segment slot of U_k, a < k < b - 1
  auto seg_slot = [&](int64_t k, int64_t a) { return nck + (k - a - 1); };
  for (int64_t k = 0; k < n; ++k) {
    if (k % c == 0)
      push(s, STORE, k / c);
    else if (k > a_last && k < n - 1)
      push(s, STORE, seg_slot(k, a_last));
    if (k < n - 1) push(s, ADVANCE, k);
  }
  for (int64_t seg = nck - 1; seg >= 0; --seg) {
    const int64_t a = seg * c, b = (a + c < n) ? a + c : n;
    if (seg != nck - 1) {
      push(s, RESTORE, seg);
      for (int64_t k = a; k < b - 1; ++k) {
        if (k > a) push(s, STORE, seg_slot(k, a));
        push(s, ADVANCE, k);
      }
    }
    push(s, TURN, b - 1);
    for (int64_t k = b - 2; k >= a; --k) {
      push(s, RESTORE, k == a ? seg : seg_slot(k, a));
      push(s, TURN, k);
    }
  }
  *out = std::move(s);
  return true;
}

inline bool binomial(int64_t n, int64_t policy, Schedule* out) {
  if (n < 1 || n > kMaxSteps || policy > -1) return false;
  const int64_t S = (-policy < n) ? -policy : n;
  if (binomial_advances(n, S) > kMaxAdvances) return false;
  Schedule s;
  std::vector<int32_t> free_slots;                       // a stack; slot 1 is taken first
  for (int64_t j = S - 1; j >= 1; --j) free_slots.push_back((int32_t)j);
  // tasks, run last-pushed first: reverse a..b-1 from U_a (current and in snapshot `home`),
  // optionally restoring `home` first; or give snapshot `home` back
  enum Kind : int8_t { REV = 0, RESTORE_REV = 1, RELEASE = 2 };
  struct Task {
    int8_t kind;
    int64_t a, b;
    int32_t home;
  };
  std::vector<Task> todo{{REV, 0, n, 0}};
  push(s, STORE, 0);
  while (!todo.empty()) {
    const Task t = todo.back();
    todo.pop_back();
    if (t.kind == RELEASE) {
      free_slots.push_back(t.home);
      continue;
    }
    if (t.kind == RESTORE_REV) push(s, RESTORE, t.home);
    const int64_t a = t.a, b = t.b, len = b - a;
    if (len == 1) {
      push(s, TURN, a);
      continue;
    }
    const int64_t F = (int64_t)free_slots.size();
    if (F == 0) {
      for (int64_t k = b - 1; k >= a; --k) {
        if (k < b - 1) push(s, RESTORE, t.home);
        for (int64_t i = a; i < k; ++i) push(s, ADVANCE, i);
        push(s, TURN, k);
      }
      continue;
    }
    // the smallest m in [1, len-1] with f(m+1) >= f(m), f(m) = m + T(len-m, F) + T(m, F+1)
    auto f = [&](int64_t m) { return m + binomial_advances(len - m, F) + binomial_advances(m, F + 1); };
    int64_t lo = 1, hi = len - 1;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (f(mid + 1) >= f(mid))
        hi = mid;
      else
        lo = mid + 1;
    }
    const int64_t m = a + lo;
    for (int64_t i = a; i < m; ++i) push(s, ADVANCE, i);
    if (b - m == 1) {                                    // U_m is turned at once: no snapshot
      push(s, TURN, m);
      todo.push_back({RESTORE_REV, a, m, t.home});
      continue;
    }
    const int32_t j = free_slots.back();
    free_slots.pop_back();
    push(s, STORE, j);
    todo.push_back({RESTORE_REV, a, m, t.home});
    todo.push_back({RELEASE, 0, 0, j});
    todo.push_back({REV, m, b, j});
  }
  *out = std::move(s);
  return true;
}

inline bool build(int64_t n, int64_t policy, Schedule* out) {
  return policy > 0 ? equidistant(n, policy, out) : binomial(n, policy, out);
}

}  // namespace ckpt
}  // namespace acm

// rt_revolve.h -- the binomial checkpoint schedule (Griewank & Walther's
// revolve) as plain host arithmetic, with no CUDA: the runtime's reverse
// sweep takes its split points from here, and the schedule's recomputation
// count can be checked on a machine without a GPU.
//
// Reversing n time steps [l, l + n) starts from the state U^l, which is held
// (in a slot of its own) and s free checkpoint slots. With s = 0 every step
// is recomputed from U^l. Otherwise the schedule advances m steps, stores
// U^{l+m} in a free slot, reverses [l + m, l + n) with s - 1 free slots, frees
// the slot and reverses [l, l + m) with s free slots.
//
// With c = s + 1 checkpoints (the held start state counts as one), at most
// beta(c, t) = C(c + t, c) steps can be reversed when every step is advanced
// at most t times; the fewest recomputed steps for n steps with
// beta(c, t - 1) < n <= beta(c, t) is t n - beta(c + 1, t - 1). A split m
// reaches it when the right part [m, n) needs exactly t advances per step
// with c - 1 checkpoints and the left part t - 1 with c checkpoints:
//   n - beta(c - 1, t) <= m <= min(beta(c, t - 1), n - beta(c - 1, t - 1)).
// revolve_split takes the upper end of that range.
#pragma once

namespace rt {

// beta(c, t) = C(c + t, c) in double (exact while below 2^53).
inline double revolve_beta(int c, int t) {
  if (t < 0 || c < 0) return 0.0;
  double b = 1.0;
  for (int i = 1; i <= c; ++i) b = b * (t + i) / i;
  return b;
}

// Advances per step t of the optimal schedule: the smallest t with
// beta(s + 1, t) >= n.
inline int revolve_sweeps(int n, int s) {
  int t = 0;
  while (revolve_beta(s + 1, t) < (double)n) ++t;
  return t;
}

// Length m of the left part (1 <= m <= n - 1) for n >= 2 steps and s >= 1
// free slots.
inline int revolve_split(int n, int s) {
  const int c = s + 1;
  const int t = revolve_sweeps(n, s);
  double lo = (double)n - revolve_beta(c - 1, t);
  double hi = revolve_beta(c, t - 1);
  const double hi2 = (double)n - revolve_beta(c - 1, t - 1);
  if (hi2 < hi) hi = hi2;
  if (hi > (double)(n - 1)) hi = (double)(n - 1);
  if (lo < 1.0) lo = 1.0;
  const double m = hi > lo ? hi : lo;
  return (int)m;
}

// Forward steps the schedule recomputes (advances) to reverse n steps with s
// free slots: the count the runtime's reverse sweep performs.
inline long long revolve_recomputed(int n, int s) {
  if (n <= 1) return 0;
  if (s <= 0) return (long long)n * (n - 1) / 2;
  const int m = revolve_split(n, s);
  return m + revolve_recomputed(n - m, s - 1) + revolve_recomputed(m, s);
}

// Griewank & Walther's minimum t n - beta(s + 2, t - 1) for n >= 2 steps and
// s >= 0 free slots besides the held start state.
inline double revolve_optimum(int n, int s) {
  if (n <= 1) return 0.0;
  const int t = revolve_sweeps(n, s);
  return (double)t * n - revolve_beta(s + 2, t - 1);
}

}  // namespace rt

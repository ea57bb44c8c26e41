// Host check of the stagnation watch shared by the host and device loop
// tests (stall_step in mp_common.cuh): reads "window adapt n" and n errors
// from stdin, feeds them as iterations 1..n, prints the iteration at which
// the watch trips (0: never), the last low's iteration and the longest gap.
#include <cstdio>

#include "mp_common.cuh"

int main() {
  int window = 0, adapt = 0, n = 0;
  if (std::scanf("%d %d %d", &window, &adapt, &n) != 3) return 2;
  double ref_err = 0.0;
  int it_ref = 0, gap = 0, tripped = 0;
  for (int it = 1; it <= n; ++it) {
    double err = 0.0;
    if (std::scanf("%lf", &err) != 1) return 2;
    if (!tripped && mp::stall_step(err, it, window, adapt != 0, ref_err, it_ref, gap)) tripped = it;
  }
  std::printf("%d %d %d\n", tripped, it_ref, gap);
  return 0;
}

// Test driver of the library's host line search (csrc/linesearch.h, the
// state machine behind etdm_minimize, Eq. 25-29): the test process supplies
// phi(alpha) over a pipe, so the oracle's line search and this one can be run
// on the same function values.
//
// Protocol, one line each way per step (doubles printed with 17 significant
// digits, which round-trip):
//   in:  "start <E0> <d0>"
//   out: "eval <alpha>"            in: "<E> <d>"          (repeated)
//   out: "done <accepted> <trials> <alpha> <E> <d>"
// A line "quit" ends the driver.
#include <cstdio>
#include <cstring>

#include "linesearch.h"

int main() {
  char cmd[32];
  while (std::scanf("%31s", cmd) == 1) {
    if (std::strcmp(cmd, "quit") == 0) break;
    if (std::strcmp(cmd, "start") != 0) return 2;
    double E0, d0;
    if (std::scanf("%lf %lf", &E0, &d0) != 2) return 2;
    etdm::LineSearch ls;
    ls.start(E0, d0);
    while (!ls.done()) {
      std::printf("eval %.17g\n", ls.alpha());
      std::fflush(stdout);
      double E, d;
      if (std::scanf("%lf %lf", &E, &d) != 2) return 2;
      ls.feed(E, d);
    }
    const etdm::LsPoint &r = ls.result();
    if (ls.accepted())
      std::printf("done 1 %d %.17g %.17g %.17g\n", ls.trials(), r.a, r.E, r.d);
    else
      std::printf("done 0 %d 0 0 0\n", ls.trials());
    std::fflush(stdout);
  }
  return 0;
}

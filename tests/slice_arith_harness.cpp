// Host build of the FP64 form's slice arithmetic (paper_1301_0191_gb300/csrc/oz_arith.h), driven
// by tests/test_slice_arith.py: reads commands from stdin, writes results to stdout.
//   R <n> then n lines "x_1 ... x_k" as 16-hex-digit IEEE bit patterns: one operand row each;
//       prints "e" and, per entry, its kSlices digits
//   S <H> <L> <s>: prints the bit pattern of round_sum(H, L, s)
#include <cinttypes>
#include <cstdio>
#include <sstream>
#include <string>
#include <vector>
#include <iostream>

#include "oz_arith.h"

int main() {
  using namespace amb::oz;
  std::string cmd;
  while (std::cin >> cmd) {
    if (cmd == "R") {
      int n;
      std::cin >> n;
      std::string line;
      std::getline(std::cin, line);
      for (int i = 0; i < n; ++i) {
        std::getline(std::cin, line);
        std::istringstream is(line);
        std::vector<double> row;
        std::string h;
        while (is >> h) row.push_back(double_of(std::stoull(h, nullptr, 16)));
        uint64_t mx = 0;
        for (double x : row) mx = absbits(x) > mx ? absbits(x) : mx;
        const int e = mx ? exponent(mx) : 0;
        std::printf("%d", e);
        for (double x : row) {
          float d[kSlices];
          digits(x, e, d);
          for (int p = 0; p < kSlices; ++p) std::printf(" %d", (int)d[p]);
        }
        std::printf("\n");
      }
    } else if (cmd == "S") {
      long long H, L;
      int s;
      std::cin >> H >> L >> s;
      std::printf("%016" PRIx64 "\n", bits_of(round_sum(H, L, s)));
    }
  }
  return 0;
}

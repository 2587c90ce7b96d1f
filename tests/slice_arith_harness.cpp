// Host build of the FP64 form's slice arithmetic (paper_1301_0191_gb300/csrc/oz_arith.h), driven
// by tests/test_slice_arith.py: reads commands from stdin, writes results to stdout.
//   R <n> then n lines "x_1 ... x_k" as 16-hex-digit IEEE bit patterns: one operand row each;
//       prints "e" and, per entry, its kSlices digits
//   S <H> <L> <s>: prints the bit pattern of round_sum(H, L, s)
//   G <m> <n> <k> then m rows of A and n rows of B (k entries each, bit patterns): C = A B^T the way
//       the slice GEMM forms it (row exponents, digits, exact integer level sums, one rounding);
//       prints the m x n results' bit patterns row by row
#include <array>
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
    } else if (cmd == "G") {
      int m, n, k;
      std::cin >> m >> n >> k;
      auto read_rows = [&](int rows, std::vector<std::vector<double>>& v) {
        v.assign(rows, std::vector<double>(k));
        for (auto& r : v)
          for (auto& x : r) {
            std::string h;
            std::cin >> h;
            x = double_of(std::stoull(h, nullptr, 16));
          }
      };
      std::vector<std::vector<double>> A, Bm;
      read_rows(m, A);
      read_rows(n, Bm);
      // per row: exponent and digits
      auto cut = [&](const std::vector<std::vector<double>>& X, std::vector<int>& e,
                     std::vector<std::vector<std::array<int, kSlices>>>& dg) {
        e.resize(X.size());
        dg.assign(X.size(), std::vector<std::array<int, kSlices>>(k));
        for (size_t r = 0; r < X.size(); ++r) {
          uint64_t mx = 0;
          for (double x : X[r]) mx = absbits(x) > mx ? absbits(x) : mx;
          e[r] = mx ? exponent(mx) : 0;
          for (int c = 0; c < k; ++c) {
            float d[kSlices];
            digits(X[r][c], e[r], d);
            for (int p = 0; p < kSlices; ++p) dg[r][c][p] = (int)d[p];
          }
        }
      };
      std::vector<int> ea, eb;
      std::vector<std::vector<std::array<int, kSlices>>> da, db;
      cut(A, ea, da);
      cut(Bm, eb, db);
      for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
          // level sums over K (chunks of at most 256 in the kernel; exact integers below 2^24 each)
          int64_t lev[kSlices] = {0, 0, 0, 0, 0, 0, 0, 0};
          for (int c = 0; c < k; ++c)
            for (int p = 0; p < kSlices; ++p)
              for (int q = 0; p + q < kSlices; ++q) lev[p + q] += (int64_t)da[i][c][p] * db[j][c][q];
          int64_t H = 0, L = 0;
          for (int l = 0; l < 4; ++l) H = H * 128 + lev[l];
          for (int l = 4; l < 8; ++l) L = L * 128 + lev[l];
          std::printf("%s%016" PRIx64, j ? " " : "", bits_of(round_sum(H, L, ea[i] + eb[j] - 63)));
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

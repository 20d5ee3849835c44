// Prints the FP32 solve pass's launch shape (march_shape) for the grids read
// from stdin, one "nx ny nsm" per line: "strips rows chunks tasks blocks".
// Host code only; nothing runs on a GPU.
#include <cstdio>
#include "sve_march.cuh"

int main() {
  int nx, ny, nsm;
  while (std::scanf("%d %d %d", &nx, &ny, &nsm) == 3) {
    sve::DevParams P{};
    P.nx = nx;
    P.ny = ny;
    const sve::MarchShape M = sve::march_shape(P, nsm);
    std::printf("%d %d %d %lld %u\n", M.strips, M.rows, M.chunks, M.tasks, M.blocks);
  }
  return 0;
}

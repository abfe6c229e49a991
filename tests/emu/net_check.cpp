// The tensor-core forward pass of the flow initializer (initnet_tc.cuh) run
// on the host with emulated tcgen05 primitives (test infrastructure): reads
// "n blocks", the packed weights and n inputs from argv[1], runs every block
// of a persistent grid of that many blocks (each with a heap shared memory of
// exactly ntc::SMEM bytes) and writes the n x 3 outputs to argv[2].
#include "blockemu.h"
#include "initnet_tc.cuh"
#include <vector>
using namespace vio;

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[2];
  if (fread(hdr, 4, 2, f) != 2) return 2;
  const int n = hdr[0], blocks = hdr[1];
  std::vector<uint8_t> packed(net::PACKED_BYTES);
  std::vector<uint16_t> x((size_t)n * 1024);
  if (fread(packed.data(), 1, packed.size(), f) != packed.size() ||
      fread(x.data(), 2, x.size(), f) != x.size())
    return 2;
  fclose(f);
  std::vector<float> out((size_t)n * 3, -1e30f);
  int fault = 0;
  static tc::EmuTc T;
  tc::emu_tc() = &T;
  gridDim.x = blocks;
  long mmas = 0;
  for (int b = 0; b < blocks; ++b) {
    std::vector<uint8_t> smem(ntc::SMEM, 0xA5);   // garbage outside what the kernel writes
    T.smem = smem.data();
    T.smem_bytes = smem.size();
    T.mmas = 0;
    for (auto& row : T.tmem)
      for (auto& v : row) v = std::nanf("");
    const ntc::XSource src{x.data(), n, out.data()};
    emu_run_block(ntc::THREADS, [&] { ntc::run(src, packed.data(), smem.data(), &fault); },
                  EmuDim{(unsigned)b, 0, 0});
    mmas += T.mmas;
  }
  f = fopen(argv[2], "wb");
  fwrite(out.data(), 4, out.size(), f);
  fclose(f);
  printf("blocks %d samples %d mmas %ld fault %d\n", blocks, n, mmas, fault);
  return fault != 0;
}

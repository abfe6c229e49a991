// The flow network's training pass (initnet_train_dev.cuh: per-warp forward
// with the legacy mma.sync tiles, loss, FP32 backward, gradient sums in
// shared memory) run on the host with one emulated CTA (test
// infrastructure): mma.sync through the emulator's fragment layout, the
// CTA's shared memory a heap buffer of exactly train_smem_bytes(), every
// input and output its own exactly sized buffer, under AddressSanitizer.
// argv[1] holds int32 n; float32 grad_scale, radius; the packed weights
// (PACKED_BYTES); n x 1024 BF16 inputs; n x 2 float32 flows. argv[2]
// receives N_MASTER float32 gradients, then the float32 loss sum.
#include "blockemu.h"
#include "initnet_train_dev.cuh"

#include <vector>

using namespace vio;
using namespace vio::net;

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t n = 0;
  float gs = 0.f, radius = 0.f;
  if (fread(&n, 4, 1, f) != 1 || fread(&gs, 4, 1, f) != 1 || fread(&radius, 4, 1, f) != 1 ||
      n < 1)
    return 2;
  std::vector<uint8_t> packed(PACKED_BYTES);
  std::vector<uint16_t> x((size_t)n * 1024);
  std::vector<float> flow((size_t)n * 2);
  if (fread(packed.data(), 1, packed.size(), f) != packed.size() ||
      fread(x.data(), 2, x.size(), f) != x.size() ||
      fread(flow.data(), 4, flow.size(), f) != flow.size())
    return 2;
  fclose(f);
  std::vector<float> grad(N_MASTER, 0.f), loss(1, 0.f);
  std::vector<uint8_t> smem(train_smem_bytes(), 0xA5);   // garbage before the pass clears it
  gridDim.x = 1;
  emu_run_block(TRAIN_WARPS * 32, [&] {
    train_block(packed.data(), x.data(), flow.data(), nullptr, n, gs, radius, grad.data(),
                loss.data(), smem.data());
  }, EmuDim{0, 0, 0});
  f = fopen(argv[2], "wb");
  fwrite(grad.data(), 4, grad.size(), f);
  fwrite(loss.data(), 4, 1, f);
  fclose(f);
  printf("trained samples %d\n", n);
  return 0;
}

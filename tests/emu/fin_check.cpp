// The finalisation's device code (finalize_dev.cuh: survivors, occupancy,
// per-cell selection, appends, counts, statistics) run for one stream on the
// host with one emulated CTA of K3_THREADS threads (test infrastructure),
// every array in its own heap buffer of exactly its size, so that
// AddressSanitizer reports any access outside one. argv[1] holds
//   int32 W, H, cell_w, cell_h, k, cap, n0, n1, next_id, have_prev;
//   uint8 trk_status[2 cap]; float32 trk_xy[2 cap][2]; int32 list_id[2 cap];
//   int32 cand_count[cells]; uint64 cand[cells k]; uint8 spec_status[cells k];
//   float32 spec_xy[cells k][2];
// argv[2] receives int32 list_count[2]; float32 list_xy[2 cap][2];
// int32 list_id[2 cap]; uint8 list_status[2 cap]; int32 new_count;
// float32 new_xy[cap][2]; int32 next_id; uint8 occupancy[cells];
// int32 stats[VIO_N_STATS].
#include "blockemu.h"
#include "finalize_dev.cuh"

#include <vector>

using namespace vio;

template <class T>
bool rd(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return fread(v.data(), sizeof(T), n, f) == n;
}

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t h[10];
  if (fread(h, 4, 10, f) != 10) return 2;
  const int W = h[0], H = h[1], cw = h[2], ch = h[3], k = h[4], cap = h[5];
  const int cells = (W / cw) * (H / ch);
  std::vector<uint8_t> trk_status, spec_status;
  std::vector<float> trk_xy, spec_xy;
  std::vector<int32_t> list_id_in, cand_count;
  std::vector<unsigned long long> cand;
  if (!rd(f, trk_status, 2 * (size_t)cap) || !rd(f, trk_xy, 4 * (size_t)cap) ||
      !rd(f, list_id_in, 2 * (size_t)cap) || !rd(f, cand_count, cells) ||
      !rd(f, cand, (size_t)cells * k) || !rd(f, spec_status, (size_t)cells * k) ||
      !rd(f, spec_xy, 2 * (size_t)cells * k))
    return 2;
  fclose(f);

  // lists of both parities: [parity][stream 0][camera] x cap
  std::vector<float> list_xy(2 * 2 * (size_t)cap * 2, -7.f);
  std::vector<int32_t> list_id(2 * 2 * (size_t)cap, -7);
  std::vector<uint8_t> list_status(2 * 2 * (size_t)cap, 0xEE);
  std::vector<int32_t> list_count(4, -7);
  std::vector<float> new_xy(2 * (size_t)cap, -7.f);
  std::vector<int32_t> new_count(1, -7), next_id(1, h[8]), step_ctr(1, 1);
  std::vector<uint8_t> occupancy(cells, 0xEE);
  std::vector<int32_t> stats((size_t)VIO_STATS_RING * VIO_N_STATS, -7);
  for (int i = 0; i < 2 * cap; ++i) list_id[i] = list_id_in[i];   // parity 0 = input
  list_count[0] = h[6];
  list_count[1] = h[7];

  FrameLaunch fl{};
  fl.p.cell_w = cw;
  fl.p.cell_h = ch;
  fl.p.k_per_cell = k;
  fl.g.n_levels = 1;
  fl.g.w[0] = W;
  fl.g.h[0] = H;
  fl.g.pitch[0] = W;
  fl.n_streams = 1;
  fl.cap = cap;
  fl.slotted = 0;
  fl.host_parity = 0;
  fl.host_have_prev = h[9];
  fl.list_xy = list_xy.data();
  fl.list_id = list_id.data();
  fl.list_count = list_count.data();
  fl.list_status = list_status.data();
  fl.trk_xy = trk_xy.data();
  fl.trk_status = trk_status.data();
  fl.cand = cand.data();
  fl.cand_count = cand_count.data();
  fl.spec_xy = spec_xy.data();
  fl.spec_status = spec_status.data();
  fl.new_xy = new_xy.data();
  fl.new_count = new_count.data();
  fl.next_id = next_id.data();
  fl.occupancy = occupancy.data();
  fl.stats = stats.data();
  fl.step_ctr = step_ctr.data();

  std::vector<int> occ_s(cells);                  // the kernel's dynamic shared memory
  std::vector<int> ws32(K3_THREADS / 32);
  std::vector<unsigned long long> ws64(K3_THREADS / 32);
  gridDim.x = 1;
  emu_run_block(K3_THREADS, [&] { finalize_stream(fl, 0, occ_s.data(), ws32.data(), ws64.data()); },
                EmuDim{0, 0, 0});

  f = fopen(argv[2], "wb");
  fwrite(&list_count[2], 4, 2, f);
  fwrite(&list_xy[2 * 2 * (size_t)cap], 4, 4 * (size_t)cap, f);
  fwrite(&list_id[2 * (size_t)cap], 4, 2 * (size_t)cap, f);
  fwrite(&list_status[2 * (size_t)cap], 1, 2 * (size_t)cap, f);
  fwrite(new_count.data(), 4, 1, f);
  fwrite(new_xy.data(), 4, 2 * (size_t)cap, f);
  fwrite(next_id.data(), 4, 1, f);
  fwrite(occupancy.data(), 1, cells, f);
  fwrite(stats.data(), 4, VIO_N_STATS, f);   // step 1 writes ring entry 0
  fclose(f);
  printf("finalised cells %d cap %d\n", cells, cap);
  return 0;
}

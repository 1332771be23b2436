// launch.cuh -- host-side launchers of the libgbmd kernels (one per kernel family).
// Every launcher enqueues on `st` and returns the launch status; none allocates.
// Grids are tile counts: each block handles one Tile of its table.
#pragma once
#include "gbmd_internal.cuh"

namespace gbmd {

constexpr int TILE_P = 256;     // particles per block of the streaming kernels
constexpr int EV_TILE_P = 128;  // particles per FP64 energy/virial partial sum
constexpr int CELLS_PER_TILE = 8;   // warps (= cells) per block of the cell kernels
constexpr int SCAN_THREADS = 1024;

// kernel-node description for graph building: function + grid + argument values.
// Copyable: the pointer array that cudaLaunchKernel / kernel nodes want is built
// from `store` at the point of use (args_of), never kept inside the object.
struct KernelCall {
  void* func;
  dim3 grid, block;
  size_t smem;
  int nargs;
  alignas(16) unsigned char store[10][16];
};

inline void args_of(const KernelCall& k, void** a) {
  for (int i = 0; i < k.nargs; ++i) a[i] = const_cast<unsigned char*>(k.store[i]);
}

// cell list + sort + neighbour list (each a no-op for systems not rebuilding); the
// sort bins are cells, or (type, cell) pairs for systems on the tree list
KernelCall bin_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl);
KernelCall scan_call(const SysDev* d, const Tile* tiles_s, int nsys, GroupCtl* ctl);
KernelCall scatter_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl);
KernelCall cellsort_call(const SysDev* d, const Tile* tiles_c, int ntiles, GroupCtl* ctl);
KernelCall permute_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl);
KernelCall copyback_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl);
// window table of every staged 2x2x2 block (8 blocks per kernel block of 256)
KernelCall blocks_call(const SysDev* d, const Tile* tiles_b, int ntiles, GroupCtl* ctl);
KernelCall nlist_call(const SysDev* d, const Tile* tiles_c, int ntiles, GroupCtl* ctl, bool rel,
                      bool multi, bool staged);
// tree neighbour list (k_tree.cu): the boxes of every type's tree (one thread per
// leaf; tiles over the system's leaves), then the list (one thread per particle in
// cell order; tiles over particles)
KernelCall tree_build_call(const SysDev* d, const Tile* tiles_l, int ntiles, GroupCtl* ctl);
KernelCall tree_nlist_call(const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl);
// pair force kernels.  MODE_FORCE: forces at the current positions (readouts);
// MODE_EV: also energy / virial / v.v partial sums (+ per-particle arrays when the
// descriptor has them); MODE_STEP: the step kernel -- forces, the velocity Verlet
// update of every particle into the next shadow buffer, and the end-of-step
// decisions by the last of sa.total_blocks blocks over the step's force launches.
// MODE_NVT_A: the first half of an NVT step -- forces, the closing half kick and
// thermostat scaling of the previous step, v.v partial sums; the last block updates
// the thermostat.  nvt_b_call: the second half (opening scaling and kick, drift,
// shadow, rebuild check, end-of-step decisions).
enum { MODE_FORCE = 0, MODE_EV = 1, MODE_STEP = 2, MODE_NVT_A = 3 };
struct StepArgs {
  int nsys = 0;             // systems of the group (decisions of the last block)
  int total_blocks = 0;     // blocks of all the step's force launches
  cudaGraphConditionalHandle cond = 0;   // the rebuild conditional of the step graph
  int use_cond = 0;
};
// eval: the PairEval of every system of the launch
KernelCall force_call(int prec, int multi, int mode, int tpp, int block, const SysDev* d,
                      const Tile* tiles_f, int ntiles, GroupCtl* ctl, const StepArgs& sa,
                      int eval);
// staged pair force: one kernel block per 2x2x2 cell block, window in shared memory
// (mixed precision, LJ evaluator); part_base = first partial-sum slot of these tiles
KernelCall force_staged_call(int multi, int mode, const SysDev* d, const Tile* tiles_s, int ntiles,
                             GroupCtl* ctl, int part_base, int window_cap, const StepArgs& sa);
KernelCall nvt_b_call(int prec, const SysDev* d, const Tile* tiles_p, int ntiles, GroupCtl* ctl,
                      const StepArgs& sa);
constexpr int STAGED_BLOCK = 256;
// thermo reduction (K7), one block per system
KernelCall thermo_call(const SysDev* d, const Tile* tiles_s, int nsys, GroupCtl* ctl);
// import row-major tag-order staging -> internal arrays; export the reverse
KernelCall prep_state_call(const SysDev* d, const Tile* tiles_p, int ntiles, const double* pos,
                           const double* vel, int* type_by_tag, int* bad);
KernelCall import_call(const SysDev* d, const Tile* tiles_p, int ntiles, const double* pos,
                       const double* vel, const int* type, const int* image);
KernelCall export_call(const SysDev* d, const Tile* tiles_p, int ntiles, double* pos,
                       double* vel, int* image, double* force, double* pp_u, double* pp_w);
// domain decomposition (one system, d pointing at its descriptor): ghost positions
// (row-major, real units) into the current step's state; wrapped positions of listed
// tags out
KernelCall ghost_set_call(const SysDev* d, int n_ghost, const double* pos);
KernelCall gather_pos_call(const SysDev* d, const int* tags, int m, double* out);
// neighbour rows -> tag-order rows sorted ascending (test readout)
KernelCall nlist_export_call(const SysDev* d, const Tile* tiles_p, int ntiles, int* counts,
                             int* idx, int cap_out, int* too_many);

cudaError_t launch(const KernelCall& k, cudaStream_t st);

// arithmetic throughput probe (k_probe.cu): one timed launch over every SM
cudaError_t probe_run(int kind, cudaStream_t st, int iters, double* ops, float* ms);

// force-kernel variants available (threads per particle)
bool tpp_supported(int tpp);

}  // namespace gbmd

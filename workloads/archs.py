"""Architecture rows: the per-GPU limits, allocation granularities and per-class
instruction throughputs that the occupancy calculation (Eqs. 1-5) and the
instruction-mix cost (Eq. 6) take as input.

This module is pure data. It holds none of the method's arithmetic; both the
CUDA path and the CPU oracle receive a row as an input, the same way they
receive kernel descriptors.

Sources per field:

* Fermi / Kepler / Maxwell / Pascal rows: Table "GPUs used in this experiment"
  (Section III-A) for cc, multiprocessors, threads per block, warps per MP,
  blocks per MP, register file, register allocation unit, registers per
  thread and shared memory per block; Table "Instruction throughput per
  number of cycles" (Section III-B) for the per-class IPC.
  Shared memory per SM: Eq. 5 sets the per-SM amount to the per-block
  maximum S_B^cc (48 KB), and the paper's S* column (Table "Suggested
  parameters", Section IV-C: 6144 / 3072 / 1536 B = 48 KB / B*) follows from
  exactly that, so the paper rows use a single 48 KB capacity; Fermi also
  offers the 16 KB split selected by Orio's PL parameter (Fig. PerfTuning).
  Fermi allocates registers per block: with per-warp allocation the
  ATAX/Fermi row (21 registers, 192 threads, occ* = 1) could not reach
  occupancy 1.
* sm_100 / sm_103 rows: public CUDA documentation for compute capability
  10.x (64 warps and 32 blocks per SM, 64 K registers, 255 registers per
  thread, 227 KB per block, the carveout capacity set, 1 KB reserved per
  block). Fields the paper does not define (warp allocation granularity,
  shared-memory allocation unit, reserved bytes) are checked on the device
  against the CUDA occupancy API by the GPU tests.
* IPC for sm_100 / sm_103: the CUDA arithmetic-throughput table for cc 10.x;
  GB300 (sm_103) has a reduced FP64 rate (about 1.25 TFLOP/s over 152 SMs,
  i.e. 2 FP64 instructions per SM per cycle).

Instruction classes, in order: FP32, FP64, INT, GLDST (global load/store),
SLDST (shared load/store), BRANCH, SFU.
"""

CLASSES = ("FP32", "FP64", "INT", "GLDST", "SLDST", "BRANCH", "SFU")
MEM_CLASSES = ("GLDST", "SLDST")

KB = 1024


def _row(**kw):
    row = dict(
        warp_size=32,
        max_threads_block=1024,
        reg_alloc_mode=0,          # 0: per warp, 1: per block
        warp_alloc_gran=4,
        smem_reserved_block=0,
        w_sat=32,                  # warps needed to hide memory latency (model constant)
        work_scale=1024,           # K, work items per count unit (model constant)
    )
    row.update(kw)
    assert len(row["ipc"]) == 7
    assert list(row["smem_caps"]) == sorted(row["smem_caps"])
    return row


ARCHS = {
    # Fermi M2050 (Table "GPUs": cc 2, 14 MPs, 48 warps, 8 blocks, 32 K regs,
    # alloc unit 64, 63 regs/thread; Table "Instruction throughput" SM20).
    "sm_20": _row(
        name="sm_20", cc=20, n_sm=14, max_warps_sm=48, max_blocks_sm=8,
        regs_sm=32768, regs_block_max=32768, regs_thread_max=63,
        reg_alloc_unit=64, reg_alloc_mode=1, warp_alloc_gran=2,
        smem_block_max=48 * KB, smem_alloc_unit=128,
        smem_caps=[16 * KB, 48 * KB],
        ipc=[32.0, 16.0, 32.0, 16.0, 16.0, 16.0, 4.0],
    ),
    # Kepler K20 (cc 3.5, 13 MPs, 64 warps, 16 blocks, 64 K regs, unit 256).
    "sm_35": _row(
        name="sm_35", cc=35, n_sm=13, max_warps_sm=64, max_blocks_sm=16,
        regs_sm=65536, regs_block_max=65536, regs_thread_max=255,
        reg_alloc_unit=256, smem_block_max=48 * KB, smem_alloc_unit=256,
        smem_caps=[16 * KB, 32 * KB, 48 * KB],
        ipc=[192.0, 64.0, 160.0, 32.0, 32.0, 32.0, 32.0],
    ),
    # Maxwell M40 (cc 5.2, 24 MPs, 64 warps, 32 blocks).
    "sm_52": _row(
        name="sm_52", cc=52, n_sm=24, max_warps_sm=64, max_blocks_sm=32,
        regs_sm=65536, regs_block_max=65536, regs_thread_max=255,
        reg_alloc_unit=256, smem_block_max=48 * KB, smem_alloc_unit=256,
        smem_caps=[48 * KB],
        ipc=[128.0, 4.0, 64.0, 64.0, 64.0, 64.0, 32.0],
    ),
    # Pascal P100 (cc 6.0, 56 MPs, 64 warps, 32 blocks).
    "sm_60": _row(
        name="sm_60", cc=60, n_sm=56, max_warps_sm=64, max_blocks_sm=32,
        regs_sm=65536, regs_block_max=65536, regs_thread_max=255,
        reg_alloc_unit=256, smem_block_max=48 * KB, smem_alloc_unit=256,
        smem_caps=[48 * KB],
        ipc=[64.0, 32.0, 32.0, 16.0, 16.0, 16.0, 16.0],
    ),
    # B200 (cc 10.0).
    "sm_100": _row(
        name="sm_100", cc=100, n_sm=148, max_warps_sm=64, max_blocks_sm=32,
        regs_sm=65536, regs_block_max=65536, regs_thread_max=255,
        reg_alloc_unit=256, smem_block_max=227 * KB, smem_alloc_unit=128,
        smem_reserved_block=1 * KB,
        smem_caps=[0, 8 * KB, 16 * KB, 32 * KB, 64 * KB, 100 * KB, 132 * KB,
                   164 * KB, 196 * KB, 228 * KB],
        ipc=[128.0, 64.0, 64.0, 32.0, 32.0, 32.0, 16.0],
    ),
    # GB300 (cc 10.3, 152 SMs; FP64 reduced to about 2 per SM per cycle).
    "sm_103": _row(
        name="sm_103", cc=103, n_sm=152, max_warps_sm=64, max_blocks_sm=32,
        regs_sm=65536, regs_block_max=65536, regs_thread_max=255,
        reg_alloc_unit=256, smem_block_max=227 * KB, smem_alloc_unit=128,
        smem_reserved_block=1 * KB,
        smem_caps=[0, 8 * KB, 16 * KB, 32 * KB, 64 * KB, 100 * KB, 132 * KB,
                   164 * KB, 196 * KB, 228 * KB],
        ipc=[128.0, 2.0, 64.0, 32.0, 32.0, 32.0, 16.0],
    ),
}


def arch(name):
    """Return a copy of one architecture row by name ("sm_20" ... "sm_103")."""
    row = ARCHS[name]
    out = dict(row)
    out["smem_caps"] = list(row["smem_caps"])
    out["ipc"] = list(row["ipc"])
    return out

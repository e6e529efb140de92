"""Helpers for the GPU parity tests (CUDA library vs FP64 oracle)."""
import numpy as np

from paper_1001_0599_gb300 import synthetic

# Relative L2 tolerance of one projector call in FP32 against the FP64 oracle,
# and of a reconstruction after a fixed iteration count.
TOL_CALL = 1e-5
TOL_RECON = 1e-4


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def host(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x) -> np.ndarray:
    """Round an FP64 array to the FP32 values both sides consume."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


# Geometries spanning several tiles and ragged tails (sizes that are not
# multiples of the kernels' tiles), nu != nv, single view, one-slice and
# one-row cases, short scans and anisotropic voxels.
CASES = {
    "small": synthetic.workload("small"),
    "odd": synthetic.Workload("odd", 13, 11, 9, 1.7, 1.3, 2.1, 37, 23, 1.1, 0.9, 7, sad=300.0, sdd=480.0,
                              arc_deg=200.0),
    "one_view": synthetic.Workload("one_view", 20, 18, 70, 1.0, 1.0, 0.5, 40, 96, 0.7, 0.4, 1,
                                   sad=200.0, sdd=350.0),
    "one_slice": synthetic.Workload("one_slice", 33, 29, 1, 1.0, 1.0, 1.0, 50, 3, 1.0, 1.0, 5,
                                    sad=150.0, sdd=220.0),
    "one_row": synthetic.Workload("one_row", 24, 24, 10, 1.0, 1.0, 1.0, 45, 1, 0.9, 0.9, 6,
                                  sad=150.0, sdd=230.0),
    "tall": synthetic.Workload("tall", 16, 16, 130, 2.0, 2.0, 0.8, 30, 140, 1.5, 1.2, 4, sad=400.0,
                               sdd=600.0),
    # exactly 1024 detector rows: the tallest detector of the sheet projector (8 rows per thread)
    "rows_1024": synthetic.Workload("rows_1024", 8, 10, 180, 2.0, 2.0, 0.45, 11, 1024, 2.2, 0.33, 3,
                                    sad=300.0, sdd=450.0),
    # z tents over 17-20 detector rows: the transpose's long-tent (interval-sum) variant
    "long_tent": synthetic.Workload("long_tent", 24, 24, 40, 2.0, 2.0, 2.0, 48, 160, 1.5, 0.4, 5,
                                    sad=500.0, sdd=750.0),
    # a fine, wide detector: the transpose's staged patch exceeds shared memory and
    # rows are read from global memory (unstaged path)
    "unstaged": synthetic.Workload("unstaged", 16, 16, 12, 2.0, 2.0, 2.0, 1200, 40, 0.04, 0.5, 3,
                                   sad=300.0, sdd=450.0),
    # a single voxel
    "single_voxel": synthetic.Workload("single_voxel", 1, 1, 1, 2.0, 2.0, 2.0, 9, 7, 1.0, 1.0, 3,
                                       sad=100.0, sdd=150.0),
    # ragged bricks along y and z on a grid the ROF kernel stages with tensor copies
    # (z a multiple of 4 and at least the 40-slice staging box)
    "ragged_tma": synthetic.Workload("ragged_tma", 40, 36, 44, 1.0, 1.0, 1.0, 64, 48, 1.2, 1.2, 6, sad=300.0,
                                     sdd=450.0),
    # more than 1024 detector rows: exercises the warp-per-column projector variant
    "very_tall": synthetic.Workload("very_tall", 10, 9, 300, 2.0, 2.0, 0.3, 9, 1100, 2.5, 0.35, 2,
                                    sad=300.0, sdd=450.0),
}


def geometries(name):
    from oracle import oracle as orc
    from paper_1001_0599_gb300 import cbct
    wl = CASES[name]
    return wl, cbct.geometry_from_workload(wl), orc.Geometry.from_workload(wl)

"""Small, fixed workloads for profiling single kernels of libkrpls with ncu.

  python -m paper_2301_12584_gb300.profile_cases descent   # krp_descent_fast, N=3, I=2^20, R=32, J=2^16
  python -m paper_2301_12584_gb300.profile_cases descent_exact # the same draws in the exact-decision mode
  python -m paper_2301_12584_gb300.profile_cases build     # tree_leaves_fp32, one factor 2^21 x 32
  python -m paper_2301_12584_gb300.profile_cases build_tc  # tree_leaves_tc (BF16x3 on tcgen05), same factor
  python -m paper_2301_12584_gb300.profile_cases build_exact # exactly accumulated leaves + build_dtop, same factor
  python -m paper_2301_12584_gb300.profile_cases prep      # prep_pinv / prep_eig, R=32, N=3
  python -m paper_2301_12584_gb300.profile_cases descent64 # krp_descent<64,2> (team kernel), N=4, I=2^18, J=2^15
  python -m paper_2301_12584_gb300.profile_cases descent100 # team descent (default form), N=3, I=2^20, R=100, J=2^14
  python -m paper_2301_12584_gb300.profile_cases descent100_nm # krp_descent_nm<128> (node-major form), same case
  python -m paper_2301_12584_gb300.profile_cases build100   # tree_leaves_fp32, one factor 2^20 x 100
  python -m paper_2301_12584_gb300.profile_cases build100_tc # tree_leaves_tc_pipe<128,.> (BF16x3), same factor
  python -m paper_2301_12584_gb300.profile_cases prep100    # prep_pinv / prep_eig / prep_etree, R=100, N=3
  python -m paper_2301_12584_gb300.profile_cases minv100    # apply_minv<128>: U_0 = Y M⁻¹, 2^21 x 100
  python -m paper_2301_12584_gb300.profile_cases rank_tc64 # tensor-core node-major draw, N=4, I=2^20, R=64, J=2^17
  python -m paper_2301_12584_gb300.profile_cases rank_tc128 # the same at R=128
  python -m paper_2301_12584_gb300.profile_cases peaks      # FP32 / FP64 FMA and L2 read throughput probes

Each case runs its kernel a few times (the first launches warm up), checks the
device status and exits 0.  Inputs are the seeded generators of synth.py.
"""
import sys

import torch

from . import synth
from .krpls import Sampler


def descent(precision=0):
    I, R, J = 1 << 20, 32, 1 << 16
    Us = synth.skewed_row_factors(3, I, R, seed=0)
    s = Sampler([I] * 3, R, 32, precision)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    idx = torch.zeros((3, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    SA = torch.zeros((J, R), device="cuda")
    for d in range(3):
        s.sample(-1, J, 1, d, idx, w, None, SA)
    assert s.sync_status() == 0, s.last_error()


def descent64():
    I, R, J = 1 << 18, 64, 1 << 15
    Us = synth.uniform_factors(4, I, R, seed=0)
    s = Sampler([I] * 4, R, R)
    for k in range(4):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    idx = torch.zeros((4, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    for d in range(3):
        s.sample(-1, J, 1, d, idx, w)
    assert s.sync_status() == 0, s.last_error()


def descent100(form=0):
    I, R, J = 1 << 20, 100, 1 << 14
    Us = synth.gaussian_factors(3, I, R, seed=0)
    s = Sampler([I] * 3, R, R)
    s.set_descent_form(form)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    idx = torch.zeros((3, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    SA = torch.zeros((J, R), device="cuda")
    for d in range(3):
        s.sample(0, J, 1, d, idx, w, None, SA)
    assert s.sync_status() == 0, s.last_error()


def rank_tc(R=64, form=3, draws=2):
    """The rank sweep's draw (N=4, I=2^20, F=R, J=2^17) in the tensor-core
    node-major form (form 3) or another form."""
    N, I, J = 4, 1 << 20, 1 << 17
    Us = synth.uniform_factors(N, I, R, seed=0)
    s = Sampler([I] * N, R, R)
    s.set_descent_form(form)
    for k in range(N):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    idx = torch.zeros((N, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    SA = torch.zeros((J, R), device="cuda")
    s.sample_prepare(-1)
    for d in range(draws):
        s.sample_draw(-1, J, 1, d, idx, w, None, SA)
    assert s.sync_status() == 0, s.last_error()


def build(precision=0, I=1 << 21, R=32):
    U = torch.from_numpy(synth.skewed_row_factors(1, I, R, seed=0)[0]).cuda()
    s = Sampler([I], R, R, precision)
    for _ in range(3):
        s.set_factor(0, U)
    assert s.sync_status() == 0, s.last_error()


def build_tc():
    build(precision=1)


def prep100():
    I, R = 1 << 14, 100
    Us = synth.gaussian_factors(3, I, R, seed=0)
    s = Sampler([I] * 3, R, R)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    for _ in range(4):
        s.sample_prepare(0)
    assert s.sync_status() == 0, s.last_error()


def minv100():
    from .krpls import SparseTensor
    dims, R, J = (1 << 21, 64, 64), 100, 1 << 14
    coords, vals = synth.sparse_zipf_tensor(dims, 200000, seed=0)
    Us = synth.gaussian_factors(3, list(dims), R, seed=1)
    s = Sampler(list(dims), R, R)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    t = SparseTensor(dims, coords, vals)
    idx = torch.zeros((3, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    SA = torch.zeros((J, R), device="cuda")
    Uo = torch.zeros((dims[0], R), device="cuda")
    for d in range(3):
        s.sample(0, J, 1, d, idx, w, None, SA)
        s.solve_sparse(t, 0, J, idx, w, SA, Uo)
    assert s.sync_status() == 0, s.last_error()


def minv100_tc():
    """minv100 with a BF16x3 sampler: Y M^-1 on the tensor cores (TF32x3)."""
    from .krpls import SparseTensor
    dims, R, J = (1 << 21, 64, 64), 100, 1 << 14
    coords, vals = synth.sparse_zipf_tensor(dims, 200000, seed=0)
    Us = synth.gaussian_factors(3, list(dims), R, seed=1)
    s = Sampler(list(dims), R, R, 1)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    t = SparseTensor(dims, coords, vals)
    idx = torch.zeros((3, J), dtype=torch.int32, device="cuda")
    w = torch.zeros(J, device="cuda")
    SA = torch.zeros((J, R), device="cuda")
    Uo = torch.zeros((dims[0], R), device="cuda")
    for d in range(3):
        s.sample(0, J, 1, d, idx, w, None, SA)
        s.solve_sparse(t, 0, J, idx, w, SA, Uo)
    assert s.sync_status() == 0, s.last_error()


def sweep25(precision=0, nnz=20_000_000, sweeps=3, R=25):
    """STS-CP sweeps (Alg. 6) at rank R (25 by default), J = 2^16 on the
    2^22 x 2^22 x 2^14 Zipf tensor with nnz nonzeros (generated on the
    device), from the benchmark's data-aware start."""
    import numpy as np
    from .krpls import SparseTensor
    dims, J = (1 << 22, 1 << 22, 1 << 14), 1 << 16
    coords, vals = synth.sparse_zipf_tensor(dims, nnz, seed=0, device=torch.device("cuda"))
    t = SparseTensor(dims, coords, vals)
    Us = synth.gaussian_factors(3, list(dims), R, seed=0)
    s = Sampler(list(dims), R, 0, precision)
    for k in range(3):
        cnt = np.bincount(coords[k], minlength=dims[k]).astype(np.float64) + 0.01
        sc = np.sqrt(cnt / cnt.mean()).astype(np.float32)
        s.set_factor(k, torch.from_numpy(Us[k] * sc[:, None]).cuda())
    from .krpls import launch_count
    sigma = torch.zeros(R, device="cuda")
    n0 = launch_count()
    for sw in range(sweeps):
        s.cp_als_sweep(t, J, 1, 3 * sw, sigma)
        if sw == 0:
            print("launches per sweep:", launch_count() - n0)
    assert s.sync_status() == 0, s.last_error()


def prep():
    I, R = 1 << 16, 32
    Us = synth.skewed_row_factors(3, I, R, seed=0)
    s = Sampler([I] * 3, R, 32)
    for k in range(3):
        s.set_factor(k, torch.from_numpy(Us[k]).cuda())
    for _ in range(4):
        s.sample_prepare(-1)
    assert s.sync_status() == 0, s.last_error()


def probe_peaks():
    """FP32 (scalar, paired), FP64 TFLOP/s and L2 read GB/s of the current
    device, from libkrpprobe.so (measure/probe.cu)."""
    import ctypes as C
    import os
    lib = C.CDLL(os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkrpprobe.so"))
    lib.krp_probe_peaks.restype = C.c_int
    lib.krp_probe_peaks.argtypes = [C.c_void_p, C.c_void_p]
    out = (C.c_double * 4)()
    code = lib.krp_probe_peaks(C.cast(out, C.c_void_p), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if code != 0:
        raise RuntimeError(f"krp_probe_peaks failed ({code})")
    return {"fp32_tflops": out[0], "fp32x2_tflops": out[1], "fp64_tflops": out[2], "l2_read_gbs": out[3]}


def peaks():
    import json
    print(json.dumps(probe_peaks()))


if __name__ == "__main__":
    {"descent": descent, "descent_exact": lambda: descent(2), "build_exact": lambda: build(2),
     "descent64": descent64, "descent100": descent100,
     "descent100_nm": lambda: descent100(2), "build": build, "build_tc": build_tc,
     "build100": lambda: build(0, 1 << 20, 100), "build100_tc": lambda: build(1, 1 << 20, 100),
     "prep": prep, "prep100": prep100, "minv100": minv100, "minv100_tc": minv100_tc, "sweep25": sweep25,
     "sweep100_bf16x3": lambda: sweep25(precision=1, R=100),
     "sweep100_bf16x3_2e8": lambda: sweep25(precision=1, nnz=200_000_000, R=100),
     "rank_tc64": lambda: rank_tc(64), "rank_tc128": lambda: rank_tc(128),
     "peaks": peaks}[sys.argv[1]]()
    torch.cuda.synchronize()
    print("ok")

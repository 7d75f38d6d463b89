"""The allocation-free conserved-sums entry point against the context one.

fargo_sums_noalloc serves callers that cannot allocate device memory
themselves (their device memory belongs to another allocator, or they cannot
afford the implicit synchronisation of cudaMalloc/cudaFree).  This file is
collected last so that a failure here leaves every other test already run;
it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import make_ctx

pytestmark = pytest.mark.gpu

# (name, workload factory, per-ring frame term passed by the caller)
#   "none": NULL, the library forms R^2 Omega_f (cylindrical, spherical);
#   "zero": a plain Cartesian box carries no frame term whatever its Omega_f;
#   "sheet": the shearing sheet's 2 Omega_f y.
CASES = [
    ("sph3d", lambda: W.random_box(W.SPH, 64, 24, 14, g=3, seed=21, nu=1e-3, planet=False), "none"),
    ("cyl2d-iso", lambda: W.random_box(W.CYL, 70, 33, 1, g=3, seed=21, iso=True, nu=1e-3, planet=False), "none"),
    ("cart2d", lambda: W.random_box(W.CART, 37, 21, 1, g=3, seed=21, nu=1e-3, planet=False), "zero"),
    ("sph3d-rotating", lambda: W.random_box(W.SPH, 40, 20, 10, g=3, seed=22, nu=1e-3, planet=False,
                                            omega_f=0.7), "none"),
    ("cyl2d-rotating", lambda: W.random_box(W.CYL, 70, 33, 1, g=3, seed=23, iso=True, nu=1e-3, planet=False,
                                            omega_f=-0.4), "none"),
    ("cart2d-rotating", lambda: W.random_box(W.CART, 37, 21, 1, g=3, seed=24, nu=1e-3, planet=False,
                                             omega_f=0.9), "zero"),
    ("shearing-sheet", lambda: W.perturb(W.shearing_sheet(nx=40, ny=48, omega=1.3), seed=25, amp=1e-2), "sheet"),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sums_without_allocation_match_context_sums(case, precision):
    import torch
    import paper_1602_02359_b300 as fb
    _, make, frame = case
    w = make()
    c = make_ctx(w, precision)
    want = c.sums()
    dt = torch.float64 if precision == fb.F64 else torch.float32
    dev = torch.device("cuda", torch.cuda.current_device())
    fields = {k: torch.empty(w.shape, dtype=dt, device=dev) for k in ("rho", "e", "vx")}
    for k, t in fields.items():
        c.get_field(k, out=t)
    torch.cuda.synchronize()
    # volume and lever arm per ring, from the geometry of the mesh
    _, _, _, _, vol, dxr = oracle.Oracle(w).geometry()
    dx = (w.xmax - w.xmin) / w.nx
    vol_t = torch.tensor(np.ascontiguousarray(vol[:w.nz_t, :w.ny_t]), dtype=torch.float64, device=dev)
    R_t = torch.tensor(np.ascontiguousarray(dxr[:w.nz_t, :w.ny_t] / dx), dtype=torch.float64, device=dev)
    wf = None
    if frame == "zero":
        wf = torch.zeros((w.nz_t, w.ny_t), dtype=torch.float64, device=dev)
    elif frame == "sheet":
        ym = W.centres(np.asarray(w.yf))[:w.ny_t]
        wf = torch.tensor(np.broadcast_to(2.0 * w.omega_f * ym, (w.nz_t, w.ny_t)).copy(), dtype=torch.float64,
                          device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share the scratch array
        out.zero_()
        fb.sums_noalloc(fields["rho"], None if w.iso else fields["e"], fields["vx"], precision, w.nx, w.ny, w.nz,
                        w.g, vol_t, R_t, w.omega_f, out, stream=stream, wframe=wf)
        torch.cuda.current_stream().synchronize()
        got = out.cpu().numpy()
        for a, b in zip(got, want):
            assert abs(a - b) <= 1e-14 * max(abs(b), 1e-300) + 1e-300, (got, want)
    c.close()


def test_block_count_beyond_the_scratch_is_rejected():
    import torch
    import paper_1602_02359_b300 as fb
    dev = torch.device("cuda", torch.cuda.current_device())
    a = torch.zeros((2, 2, 8), dtype=torch.float64, device=dev)
    r = torch.ones((1, 1), dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    with pytest.raises(fb.FargoError) as e:
        fb.sums_noalloc(a, a, a, fb.F64, 8, 1, 1, 0, r, r, 0.0, out, nblocks=1185)
    assert e.value.code == -6

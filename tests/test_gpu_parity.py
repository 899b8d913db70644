"""GPU parity: the CUDA step (through the C ABI) against the FP64 oracle on the
same seeded float32 inputs, element by element.

Tolerances (relative L2 of phi after the configured steps, and the same
bound on the per-element error max |delta phi| / max |phi|):
  FP32 state            <= 1e-5
  FP16 / BF16 offsets   <= 2e-3
Grids are ragged (nx not a multiple of the 256-thread row block) and span
several blocks and rows; walls, velocity kinds and storage forms are crossed.
Most cases add a positive background to the hill (so that every node carries
signal); the cases of test_kernels_without_background run the hill alone, so
that neither norm is diluted by a background and the dilute tails and the wall
rows count in full.
"""
import numpy as np
import pytest

from _common import Case, assert_parity, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 2e-3}

CASES_2D = [
    Case(storage="f32"),
    Case(storage="f32", ukind="none", sched=False),
    Case(storage="f32", ukind="field", sched=False, nx=257, ny=41),
    Case(storage="f32", bc=("noflux", "noflux"), ukind="row", ny=33),
    Case(storage="f32", bc=("noflux", "noflux"), ukind="field"),
    Case(storage="f32", bc=("bounceback", "bounceback"), ukind="field"),
    Case(storage="f32", bc=("dirichlet", "dirichlet"), phi_w=(1.0, 0.25), ukind="field"),
    Case(storage="f32", bc=("noflux", "bounceback"), ukind="row"),
    Case(storage="f16"),
    Case(storage="bf16"),
    Case(storage="f16", bc=("noflux", "noflux"), ukind="row", ny=33),
    Case(storage="bf16", bc=("bounceback", "bounceback"), ukind="field"),
    Case(storage="f16", bc=("dirichlet", "dirichlet"), phi_w=(1.0, 0.25), ukind="field"),
    Case(storage="f32", nx=1, ny=5, ukind="none", sched=False, steps=50),
    Case(storage="f32", model="B1", umax=0.1),
    Case(storage="f32", model="B2", umax=0.1, bc=("noflux", "noflux"), ukind="row"),
    Case(storage="f32", model="B3", umax=0.1, bc=("bounceback", "bounceback")),
    Case(storage="bf16", model="B3"),
    Case(storage="f32", nx=33, ny=1, ukind="field", steps=50),
]

CASES_3D = [
    Case(lattice=15, nx=40, ny=23, nz=17, steps=60, D=np.array([[0.03, 0.005, -0.004],
                                                                [0.005, 0.025, 0.003],
                                                                [-0.004, 0.003, 0.035]])),
    Case(lattice=15, nx=40, ny=23, nz=17, steps=60, bc=("noflux", "noflux"), ukind="row",
         D=np.diag([0.02, 0.03, 0.04])),
    Case(lattice=15, nx=33, ny=19, nz=11, steps=60, bc=("bounceback", "bounceback"),
         D=np.diag([0.02, 0.03, 0.04])),
    Case(lattice=15, nx=40, ny=23, nz=17, steps=60, storage="f16", D=np.diag([0.03, 0.02, 0.04])),
    Case(lattice=15, nx=40, ny=23, nz=17, steps=60, storage="bf16", D=np.diag([0.03, 0.02, 0.04])),
]


def _id(c):
    return f"q{c.lattice}-{c.model}-{c.storage}-{c.bc[0]}-{c.bc[1]}-{c.ukind}-{c.nx}x{c.ny}x{c.nz}"


@pytest.mark.parametrize("case", CASES_2D + CASES_3D, ids=_id)
def test_step_matches_oracle(O, case):
    phi0, a, sched = case.inputs()
    got, s = run_gpu(case, phi0, a, sched)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[case.storage])
    if case.bc[0] == "dirichlet":
        assert np.abs(got[0] - case.phi_w[0]).max() < 1e-5
        assert np.abs(got[-1] - case.phi_w[1]).max() < 1e-5


# (storage, walls, velocity kind, launch (block, vec) or None for the default one-node kernel)
NOBG = [
    ("f32", ("periodic", "periodic"), "field", None),
    ("f32", ("noflux", "noflux"), "row", None),
    ("f32", ("bounceback", "bounceback"), "field", (64, 6)),
    ("bf16", ("periodic", "periodic"), "field", None),
    ("f16", ("noflux", "noflux"), "row", (64, 5)),
    ("bf16", ("bounceback", "bounceback"), "field", (64, 6)),
    ("f16", ("periodic", "periodic"), "field", (128, 7)),
    ("bf16", ("noflux", "noflux"), "row", (128, 8)),
]


@pytest.mark.parametrize("storage,bc,ukind,launch", NOBG,
                         ids=lambda v: "-".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_kernels_without_background(O, storage, bc, ukind, launch):
    """The hill alone (phi from 1 down to ~1e-14 in the corners) on each kernel
    family: one-node, node-quad (vec 6), node-pair (vec 5) and TMA-staged (vec 7,
    8), with periodic, Neumann and bounce-back walls; relative L2 and per-element
    bounds, and the wall rows on their own."""
    case = Case(storage=storage, bc=bc, ukind=ukind, nx=512, ny=40, steps=120, bg=False)
    phi0, a, sched = case.inputs()
    if launch is None:
        got, _ = run_gpu(case, phi0, a, sched)
    else:
        got, s = _run_vec3(case, phi0, a, sched, vec=launch[1], block=launch[0])
        s.sync()
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    if bc[0] != "periodic":
        walls = np.array([0, case.ny - 1])
        assert np.abs(got[walls] - want[walls]).max() <= TOL[storage] * np.abs(want).max()


@pytest.mark.parametrize("storage,launch", [("f32", None), ("bf16", (64, 5)), ("f16", (64, 5)),
                                            ("bf16", (256, 9)), ("f16", (256, 9))])
def test_d3q15_without_background(O, storage, launch):
    """D3Q15 hill alone (one-node FP32 kernel, node-pair and z-walk 16-bit
    kernels), Neumann walls on the y faces; relative L2 and per-element bounds."""
    nx, ny = (64, 24) if launch and launch[1] == 9 else (40, 23)
    case = Case(lattice=15, storage=storage, nx=nx, ny=ny, nz=17, steps=60, bc=("noflux", "noflux"),
                D=np.diag([0.02, 0.03, 0.04]), bg=False)
    phi0, a, sched = case.inputs()
    if launch is None:
        got, _ = run_gpu(case, phi0, a, sched)
    else:
        got, _ = _run_vec3(case, phi0, a, sched, vec=launch[1], block=launch[0])
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])


BOX = [
    # (lattice, storage, x faces, y faces, z faces)
    (9, "f32", ("noflux", "noflux"), ("periodic", "periodic"), None),
    (9, "f32", ("bounceback", "bounceback"), ("periodic", "periodic"), None),
    (9, "f32", ("noflux", "noflux"), ("bounceback", "bounceback"), None),
    (9, "f32", ("bounceback", "bounceback"), ("noflux", "noflux"), None),
    (9, "f32", ("bounceback", "noflux"), ("dirichlet", "dirichlet"), None),
    (9, "bf16", ("noflux", "noflux"), ("noflux", "noflux"), None),
    (9, "f16", ("bounceback", "bounceback"), ("bounceback", "bounceback"), None),
    (15, "f32", ("periodic", "periodic"), ("periodic", "periodic"), ("noflux", "noflux")),
    (15, "f32", ("bounceback", "bounceback"), ("noflux", "noflux"), ("bounceback", "bounceback")),
    (15, "bf16", ("noflux", "noflux"), ("bounceback", "bounceback"), ("noflux", "noflux")),
]


@pytest.mark.parametrize("lattice,storage,bcx,bcy,bcz", BOX,
                         ids=lambda v: "-".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_walls_on_x_and_z_faces(O, lattice, storage, bcx, bcy, bcz):
    """Walls on two and on four (six) faces, with a velocity field and a
    schedule: the general box kernel against the oracle, whose x and z walls are
    pinned against its y walls by the axis exchange (tests/test_oracle_walls.py).
    With bounce-back on every face the total is conserved."""
    kw = dict(bc=bcy, bc_x=bcx, phi_w=(1.0, 0.25) if bcy[0] == "dirichlet" else (0.0, 0.0))
    if lattice == 9:
        case = Case(storage=storage, nx=37, ny=29, steps=80, **kw)
    else:
        case = Case(lattice=15, storage=storage, nx=19, ny=13, nz=11, steps=40, D=D3, bc_z=bcz, **kw)
    phi0, a, sched = case.inputs()
    got, s = run_gpu(case, phi0, a, sched)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    if all(b[0] in ("bounceback", "periodic") for b in (bcx, bcy, bcz or ("periodic",))):
        m = s.sum_phi()
        assert abs(m - phi0.astype(np.float64).sum()) <= {"f32": 1e-6, "f16": 1e-4, "bf16": 1e-3}[storage] * m
    s.close()


@pytest.mark.parametrize("vec,block", [(1, 64), (2, 128)])
def test_launch_shapes_agree(vec, block):
    """The same step under other launch shapes gives the identical result."""
    import torch
    from paper_1404_2363_gb300.solver import Solver

    case = Case(storage="f32")
    phi0, a, sched = case.inputs()
    ref, _ = run_gpu(case, phi0, a, sched)
    s = Solver(nx=case.nx, ny=case.ny)
    s.set_launch(block=block, vec=vec)
    s.set_D(case.D)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(case.steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref)


def test_config1_gaussian_hill_full(O):
    """The anisotropic Gaussian hill of the first workload at its full size and
    length: 128 x 128 periodic, u = 0, 1000 steps, FP32 vs FP64 oracle."""
    from paper_1404_2363_gb300 import workloads as W

    wl = W.gaussian_workload(128)
    case = Case(nx=128, ny=128, ukind="none", sched=False, steps=1000, D=wl["D"])
    phi0 = wl["phi0"].astype(np.float32)
    got, s = run_gpu(case, phi0, None, None)
    want = run_oracle(O, case, phi0, None, None)
    assert_parity(got, want, 1e-5)
    # FP64 conservation check on the device
    assert abs(s.sum_phi() - phi0.astype(np.float64).sum()) / phi0.sum() < 1e-5


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("bc,ukind", [(("periodic", "periodic"), "field"), (("noflux", "noflux"), "row"),
                                      (("bounceback", "bounceback"), "field"),
                                      (("dirichlet", "dirichlet"), "field"), (("periodic", "periodic"), "none")])
def test_pair_offset_kernel(O, storage, bc, ukind):
    """The node-pair kernel of the 16-bit forms (launch vec = 5, paired FP32
    arithmetic) against the oracle on a 302 x 37 grid (151 pairs per row: ragged
    64-thread blocks), and against the one-node kernel: the same operations, up to
    the compiler's fusing of paired multiply-adds, so the fields agree to the
    16-bit rounding of a few offsets."""
    case = Case(storage=storage, bc=bc, ukind=ukind, sched=ukind != "none", nx=302, ny=37,
                phi_w=(1.0, 0.25) if bc[0] == "dirichlet" else (0.0, 0.0))
    phi0, a, sched = case.inputs()
    got, _ = _run_vec3(case, phi0, a, sched, vec=5, block=64)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    one, _ = _run_vec3(case, phi0, a, sched, vec=1, block=64)
    assert rel_l2(got, one) <= TOL[storage] / 4
    if ukind != "field":   # no products with a varying velocity: nothing to fuse differently
        assert np.array_equal(got, one)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc,ukind", [(("periodic", "periodic"), "field"), (("noflux", "noflux"), "row"),
                                      (("bounceback", "bounceback"), "field"),
                                      (("dirichlet", "dirichlet"), "field"), (("periodic", "periodic"), "none")])
def test_quad_kernel(O, storage, bc, ukind):
    """The node-quad kernel (launch vec = 6: four nodes per thread, 128-bit FP32 /
    64-bit 16-bit vector loads and stores, warp shuffles for the shifted pulls)
    against the oracle on a 300 x 37 grid (75 quads per row: ragged 64-thread
    blocks and a partial warp at the seam), and against the one-node kernel."""
    case = Case(storage=storage, bc=bc, ukind=ukind, sched=ukind != "none", nx=300, ny=37,
                phi_w=(1.0, 0.25) if bc[0] == "dirichlet" else (0.0, 0.0))
    phi0, a, sched = case.inputs()
    got, _ = _run_vec3(case, phi0, a, sched, vec=6, block=64)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    one, _ = _run_vec3(case, phi0, a, sched, vec=1, block=64)
    assert rel_l2(got, one) <= TOL[storage] / 4


@pytest.mark.parametrize("nx,ny", [(4, 6), (8, 5), (132, 9)])
def test_quad_kernel_narrow_grids(O, nx, ny):
    """One quad per row (both shuffle partners are fix-up loads across the
    periodic seam), two quads, and 33 quads (a warp edge inside the row)."""
    for storage in ("f32", "bf16"):
        case = Case(storage=storage, nx=nx, ny=ny, steps=40)
        phi0, a, sched = case.inputs()
        got, _ = _run_vec3(case, phi0, a, sched, vec=6, block=32)
        want = run_oracle(O, case, phi0, a, sched)
        assert_parity(got, want, TOL[storage], (storage, nx, ny))


@pytest.mark.parametrize("vec", [7, 8])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("bc,ukind", [(("periodic", "periodic"), "field"), (("noflux", "noflux"), "row"),
                                      (("bounceback", "bounceback"), "field"),
                                      (("dirichlet", "dirichlet"), "field"), (("periodic", "periodic"), "none")])
def test_tma_offset_kernel(O, storage, bc, ukind, vec):
    """The TMA-staged kernel of the D2Q9 16-bit forms (launch vec 7 / 8: source
    rows staged in shared memory by tensor copies, two or one rows per iteration)
    against the oracle on a 512 x 37 grid (74 strip rows: one-row work ranges), and
    against the node-pair kernel, whose arithmetic it shares."""
    case = Case(storage=storage, bc=bc, ukind=ukind, sched=ukind != "none", nx=512, ny=37,
                phi_w=(1.0, 0.25) if bc[0] == "dirichlet" else (0.0, 0.0))
    phi0, a, sched = case.inputs()
    got, s = _run_vec3(case, phi0, a, sched, vec=vec, block=128)
    s.sync()
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    pair, _ = _run_vec3(case, phi0, a, sched, vec=5, block=64)
    assert rel_l2(got, pair) <= TOL[storage] / 4


@pytest.mark.parametrize("nx,ny,steps", [(768, 600, 12), (256, 1, 30), (256, 3, 30), (1024, 5, 20)])
def test_tma_kernel_work_ranges(O, nx, ny, steps):
    """Row ranges of odd and even lengths (768 x 600: three strips), a one-row and
    a three-row periodic grid (every staged row wraps), four strips of five rows."""
    for storage, vec in (("f16", 7), ("bf16", 7), ("bf16", 8)):
        case = Case(storage=storage, nx=nx, ny=ny, steps=steps)
        phi0, a, sched = case.inputs()
        got, s = _run_vec3(case, phi0, a, sched, vec=vec, block=128)
        s.sync()
        want = run_oracle(O, case, phi0, a, sched)
        assert_parity(got, want, TOL[storage], (storage, vec, nx, ny))


def test_tma_wait_timeout_is_reported_and_handle_recovers(O):
    """A zero wait limit makes every bounded wait of the TMA-staged kernel give up:
    the step reports LBM_E_TIMEOUT on the next synchronising call, no kernel hangs,
    and the same handle then runs correctly with the default limit."""
    from paper_1404_2363_gb300 import _native as N

    case = Case(storage="bf16", nx=512, ny=64, steps=20)
    phi0, a, sched = case.inputs()
    import torch
    from paper_1404_2363_gb300.solver import Solver

    s = Solver(nx=case.nx, ny=case.ny, storage="bf16")
    s.set_launch(128, 7)
    s.set_D(case.D)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.set_wait_limit(0)
    s.step(3)
    with pytest.raises(N.LbmError) as e:
        s.sync()
    assert e.value.status == N.LBM_E_TIMEOUT
    s.sync()                       # the status was cleared
    s.set_wait_limit(4_000_000_000)
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(case.steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.sync()
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL["bf16"])


D3 = np.array([[0.03, 0.005, -0.004], [0.005, 0.025, 0.003], [-0.004, 0.003, 0.035]])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("bc,ukind", [(("periodic", "periodic"), "field"), (("noflux", "noflux"), "row"),
                                      (("bounceback", "bounceback"), "field"),
                                      (("dirichlet", "dirichlet"), "field"), (("periodic", "periodic"), "none")])
def test_pair_offset_kernel_d3q15(O, storage, bc, ukind):
    """The D3Q15 node-pair kernel of the 16-bit forms (launch vec = 5: paired FP32
    decode, collision and store) against the oracle on a 70 x 13 x 9 grid (35
    pairs per row: two 32-thread blocks, the second ragged), and against the
    one-node kernel (same operations up to the folding of the schedule factor into
    the decode slopes and the compiler's fusing of paired multiply-adds)."""
    case = Case(lattice=15, storage=storage, bc=bc, ukind=ukind, sched=ukind != "none", nx=70, ny=13, nz=9,
                steps=40, D=D3, phi_w=(1.0, 0.25) if bc[0] == "dirichlet" else (0.0, 0.0))
    phi0, a, sched = case.inputs()
    got, _ = _run_vec3(case, phi0, a, sched, vec=5, block=32)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    one, _ = _run_vec3(case, phi0, a, sched, vec=1, block=64)
    assert rel_l2(got, one) <= TOL[storage] / 4
    if bc[0] == "dirichlet":
        assert np.abs(got[:, 0] - 1.0).max() < 1e-4 and np.abs(got[:, -1] - 0.25).max() < 1e-4


@pytest.mark.parametrize("nx,ny,nz", [(2, 5, 3), (4, 3, 4), (66, 4, 3)])
def test_pair_offset_kernel_d3q15_narrow_grids(O, nx, ny, nz):
    """One pair per row (both shifted pulls wrap onto the same pair), two pairs,
    and 33 pairs with 32-thread blocks (a second block of one thread)."""
    for storage in ("f16", "bf16"):
        case = Case(lattice=15, storage=storage, nx=nx, ny=ny, nz=nz, steps=30, D=D3)
        phi0, a, sched = case.inputs()
        got, _ = _run_vec3(case, phi0, a, sched, vec=5, block=32)
        want = run_oracle(O, case, phi0, a, sched)
        assert_parity(got, want, TOL[storage], (storage, nx, ny, nz))


def _run_zw(case, phi0, a, sched, planes, block=256):
    import torch
    from paper_1404_2363_gb300.solver import Solver

    s = Solver(lattice=15, nx=case.nx, ny=case.ny, nz=case.nz, storage=case.storage, bc=case.bc,
               phi_w=case.phi_w, model=case.model)
    s.set_launch(block, 9)
    s.set_zwalk(planes)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row" if case.ukind == "row" else "field")
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(case.steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.sync()
    return got


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("bc,ukind", [(("periodic", "periodic"), "field"), (("noflux", "noflux"), "row"),
                                      (("bounceback", "bounceback"), "field"),
                                      (("dirichlet", "dirichlet"), "field"), (("periodic", "periodic"), "none")])
@pytest.mark.parametrize("block", [256, 128])
def test_zwalk_offset_kernel_d3q15(O, storage, bc, ukind, block):
    """The D3Q15 z-walk kernel of the 16-bit forms (launch vec 9: 64 x 8 or 64 x 4
    tiles of the (x, y) plane walking z, phi and the velocity factors of three
    planes and the offsets of a step in shared memory) against the oracle on a
    128 x 16 x 10 grid: two tiles in x, two or four in y, z ranges of 3, 3 and 4
    planes (walks of 4 planes per CTA asked), and against the node-pair kernel,
    whose arithmetic it shares."""
    case = Case(lattice=15, storage=storage, bc=bc, ukind=ukind, sched=ukind != "none", nx=128, ny=16, nz=10,
                steps=30, D=D3, phi_w=(1.0, 0.25) if bc[0] == "dirichlet" else (0.0, 0.0))
    phi0, a, sched = case.inputs()
    got = _run_zw(case, phi0, a, sched, planes=4, block=block)
    want = run_oracle(O, case, phi0, a, sched)
    assert_parity(got, want, TOL[storage])
    pair, _ = _run_vec3(case, phi0, a, sched, vec=5, block=64)
    assert rel_l2(got, pair) <= TOL[storage] / 4
    if bc[0] == "dirichlet":
        assert np.abs(got[:, 0] - 1.0).max() < 1e-4 and np.abs(got[:, -1] - 0.25).max() < 1e-4


@pytest.mark.parametrize("nx,ny,nz,planes,steps", [(64, 8, 1, 0, 20), (64, 8, 2, 2, 20), (64, 8, 2, 1, 20),
                                                   (128, 24, 5, 0, 16), (192, 16, 7, 7, 16), (64, 40, 9, 2, 12)])
def test_zwalk_d3q15_work_ranges(O, nx, ny, nz, planes, steps):
    """One tile with one z plane (the three staged planes coincide, every staged
    row and column wraps), two planes walked by one CTA or by two, the launcher's
    own ranges, one walk over all seven planes (its first and last staged planes
    wrap), and five tiles in y with ranges of one and two planes; 8-row and
    4-row tiles."""
    for storage, block in (("f16", 256), ("bf16", 256), ("bf16", 128)):
        case = Case(lattice=15, storage=storage, nx=nx, ny=ny, nz=nz, steps=steps, D=D3)
        phi0, a, sched = case.inputs()
        got = _run_zw(case, phi0, a, sched, planes, block)
        want = run_oracle(O, case, phi0, a, sched)
        assert_parity(got, want, TOL[storage], (storage, block, nx, ny, nz, planes))


def test_zwalk_rejects_unsupported_shapes():
    from paper_1404_2363_gb300 import _native as N
    from paper_1404_2363_gb300.solver import Solver

    for nx, ny, storage, block in ((96, 8, "bf16", 256), (64, 12, "bf16", 256), (64, 8, "f32", 256),
                                   (64, 6, "f16", 128)):
        s = Solver(lattice=15, nx=nx, ny=ny, nz=3, storage=storage)
        with pytest.raises(N.LbmError) as e:
            s.set_launch(block, 9)
        assert e.value.status == N.LBM_E_ARG
    s = Solver(lattice=15, nx=64, ny=8, nz=3, storage="bf16")
    with pytest.raises(N.LbmError):
        s.set_launch(64, 9)
    with pytest.raises(N.LbmError):
        s.set_zwalk(-1)



def _run_vec3(case, phi0, a, sched, vec=1, block=256):
    import torch
    from paper_1404_2363_gb300.solver import Solver

    s = Solver(lattice=case.lattice, nx=case.nx, ny=case.ny, nz=case.nz, storage=case.storage, bc=case.bc,
               phi_w=case.phi_w, model=case.model)
    s.set_launch(block, vec)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row" if case.ukind == "row" else "field")
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(case.steps)
    return s.get_phi().cpu().numpy().astype(np.float64), s


def test_autotune_keeps_results(tmp_path, monkeypatch):
    """The autotuner restores the state; the tuned shape gives the same result."""
    monkeypatch.setenv("LBMCDE_TUNE_CACHE", str(tmp_path / "tune.txt"))
    import torch
    from paper_1404_2363_gb300.solver import Solver

    case = Case(storage="bf16", nx=512, ny=64, steps=30)
    phi0, a, sched = case.inputs()
    ref, _ = run_gpu(case, phi0, a, sched)
    s = Solver(nx=case.nx, ny=case.ny, storage="bf16")
    s.set_D(case.D)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    shape = s.autotune(5)
    assert s.t == 0
    s.step(case.steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    assert rel_l2(got, ref) < TOL["bf16"] / 4, shape
    # the state was restored: the tuned shape from scratch gives the same field
    again, _ = _run_vec3(case, phi0, a, sched, vec=shape[1], block=shape[0])
    assert np.array_equal(got, again), shape
    assert (tmp_path / "tune.txt").read_text().strip().endswith(f"{shape[0]} {shape[1]}")

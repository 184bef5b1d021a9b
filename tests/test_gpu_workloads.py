"""GPU parity on the workloads beyond the operator tests: the paper's plate (Sec. 4.3), the
bimaterial diffusion on a non-power-of-two grid (Sec. 4.2), several particles in one RVE,
the chemistry Newton with the full Jacobian, and the coupled adjoint under mixed
macroscopic control.  Each runs the CUDA path through the C ABI and compares fields with
the CPU oracle on the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fg_oracle as O
from paper_2411_16583_gb300 import binding as B, synth as S
from tests import test_emu_kernels as TE
from tests.helpers import TOL_STEP_FP64, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available()
    return B.load_library()


def test_bimaterial_diffusion_100(lib):
    """Sec. 4.2 type bimaterial diffusion on a 100 x 100 grid (100 = 4 x 5 x 5), two FP64
    steps against the oracle (the same case the host emulation checks)."""
    TE.test_emulated_bimaterial_diffusion_100(lib)


def test_full_chemistry_jacobian_matches_oracle(lib):
    """The chemistry Newton with the elastic part of dmu~/dc in its Jacobian, on a 32 x 32
    version of the Omega = 1.3 Saint-Venant-Kirchhoff Gumbel disc, one step."""
    TE.test_emulated_full_chemistry_jacobian_matches_oracle(lib)


def test_multi_particle_step_matches_oracle(lib):
    """Three rough particles in one 32^3 periodic RVE, each with its own influx band: one
    FP64 coupled step against the oracle."""
    w = S.multi_particle(n=32, count=3, rmin=0.12, rmax=0.17, band=2, nsteps=10,
                         phases=S.default_phases(buffer_E=S.BENCH_BUFFER_E))
    assert len(np.unique(w.phase_id)) == 2
    prm = oracle_params(w)
    ref = O.CoupledState(prm, w.c_init, w.cdot_B)
    ref.step(w.dt, np.eye(3))
    sol = B.from_workload(w, lib=lib)
    sol.step(w.dt)
    assert rel_err(sol.get(B.FIELD_F), ref.F) < TOL_STEP_FP64
    assert rel_err(sol.get(B.FIELD_C), ref.c) < TOL_STEP_FP64
    sol.close()


@pytest.mark.parametrize("ckpt", [1, 2])
def test_adjoint_under_mixed_control_matches_oracle(lib, ckpt):
    """Reverse pass of two damaging steps with F_xx under stress control on the device,
    against the oracle's adjoint (checkpoints every 1 and 2 steps)."""
    TE.test_emulated_adjoint_under_mixed_control_matches_oracle(lib, ckpt)


@pytest.mark.parametrize("shape", [(128, 128, 8), (256, 256, 16)])
def test_cluster_yzy_pass_matches_oracle(lib, shape):
    """The clustered Y-Z-Y projection pass (16-CTA clusters, tiles exchanged through
    distributed shared memory) on the device: the oracle's mechanical operator, and the
    three separate passes' result to FP32 round-off, with and without mixed control."""
    TE.test_emulated_cluster_yzy_pass_matches_oracle(lib, shape)


def test_cluster_passes_keep_the_coupled_steps(lib):
    """Two mixed coupled steps of the benchmark particle recipe at 128^3 (ny = nz = 128, so
    every FP32 Y-Z-Y chain of the mechanics and the chemistry may run clustered) with the
    clustered passes and with the three-pass chains: the same Newton iterations and fields
    equal to the solver tolerance."""
    import bench
    w = bench._workload(128, 0)
    out = []
    for cp in (1, 0):
        sol = B.from_workload(w, precision=B.FG_MIXED, lib=lib, cluster_pass=cp)
        st = [sol.step(w.dt) for _ in range(2)]
        out.append((sol.get(B.FIELD_F), sol.get(B.FIELD_C), st))
        sol.close()
    assert rel_err(out[0][0], out[1][0]) < 1e-8
    assert rel_err(out[0][1], out[1][1]) < 1e-10
    for a, b in zip(out[0][2], out[1][2]):
        assert a["newton_mech"] == b["newton_mech"] and a["newton_chem"] == b["newton_chem"]

"""Batched persistent step: every instance of a batch must evolve exactly as
the same lattice run alone through ddflb_step (same per-node arithmetic), and
the batch bookkeeping (convergence freeze, divergence, bounded barrier waits)
must behave.  One instance is also checked against the FP64 oracle directly."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D
from paper_1908_06742_gb300 import inputs
from tests.gpu_helpers import np64, rate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    D.load()


def cfg(nx, ny, bc, nu, check=10, **kw):
    w = rate(nu)
    base = dict(nx=nx, ny=ny, bc=bc, omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                omega_g=(0, w, w, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2), check_every=check)
    base.update(kw)
    return D.Config(**base)


def start_fields(c, seed):
    if c.bc == "periodic":
        F = inputs.taylor_green(c.nx, 0.02, phi_amp=0.1, ny=c.ny)
        return (F.rho, F.ux, F.uy, F.phi, F.grads)
    F = inputs.rest(c.nx, c.ny, phi=0.5 + 0.1 * seed)
    return (F.rho, F.ux, F.uy, F.phi, None)


CFGS = [cfg(40, 30, "cavity", 0.05, u_lid=0.1, phi_lid=1.0, phi_wall=0.0),
        cfg(64, 64, "periodic", 0.01),
        cfg(33, 17, "channel", 0.1, u_lid=0.05, phi_lid=2.0, phi_wall=1.0),
        cfg(130, 70, "cavity", 0.02, u_lid=0.08, phi_lid=1.0, phi_wall=0.2)]


def same(a, b):
    return torch.equal(torch.nan_to_num(a, 9.0), torch.nan_to_num(b, 9.0))


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("tiles", [(128, 1), (32, 4), (256, 1), (64, 2)])
def test_batch_equals_single_lattice_runs(tiles, schedule):
    """45 steps in chunks of 7 (graph replays plus a direct remainder launch),
    every field of every instance bit-identical to the single-lattice path;
    both schedules (persistent launch, one launch per step)."""
    steps = 45
    b = D.Batch(CFGS).set_run(tol=0.0, steps_per_launch=7).set_schedule(schedule)
    b.set_tiles(*tiles)
    assert b.schedule() == schedule
    for i, c in enumerate(CFGS):
        b.init(i, *start_fields(c, i))
    b.step(steps)
    st = b.stats()
    assert st["status"] == D.OK and not st["flags"].any()
    assert (st["state_time"] == steps).all()
    for i, c in enumerate(CFGS):
        ref = D.Lattice(c).init(*start_fields(c, i)).step(steps).fields()
        got = b.fields(i)
        for k in D.FIELD_NAMES:
            assert same(got[k], ref[k]), (i, k, tiles)
    # the residual of the last check (t = 40) matches the single path's check
    for i, c in enumerate(CFGS):
        r = D.Lattice(c).init(*start_fields(c, i)).step(40).stats()["residual"]
        assert math.isclose(st["residual"][i], r, rel_tol=1e-12), (i, st["residual"][i], r)


@pytest.mark.parametrize("schedule", [0, 1])
def test_many_tiles_per_cta(schedule):
    """One CTA per SM and a 300 x 200 cavity added: the persistent launch's
    CTAs each walk a range of tiles that crosses instances (parameters
    restaged at every change), still bit-identical to the single-lattice path;
    the per-step schedule runs the same tiles one per CTA."""
    cfgs = CFGS + [cfg(300, 200, "cavity", 0.03, u_lid=0.1, phi_lid=1.0, phi_wall=0.0)]
    steps = 23
    b = D.Batch(cfgs).set_run(tol=0.0, steps_per_launch=5).set_schedule(schedule)
    b.set_tiles(32, 4, 1)
    for i, c in enumerate(cfgs):
        b.init(i, *start_fields(c, i))
    b.step(steps)
    st = b.stats()
    assert st["status"] == D.OK and not st["flags"].any()
    for i, c in enumerate(cfgs):
        ref = D.Lattice(c).init(*start_fields(c, i)).step(steps).fields()
        got = b.fields(i)
        for k in D.FIELD_NAMES:
            assert same(got[k], ref[k]), (i, k)


@pytest.mark.parametrize("bc", ["cavity", "channel", "periodic"])
def test_single_boundary_kind_batches(bc):
    """A batch whose instances share one boundary kind runs the persistent
    kernel specialised to it; still bit-identical to the single-lattice path."""
    kw = {} if bc == "periodic" else dict(u_lid=0.08, phi_lid=1.0, phi_wall=0.2)
    cfgs = [cfg(nx, ny, bc, nu, **kw) for nx, ny, nu in ((40, 30, 0.05), (130, 70, 0.02), (64, 64, 0.01))]
    steps = 23
    b = D.Batch(cfgs).set_run(tol=0.0, steps_per_launch=5).set_schedule(0)
    for i, c in enumerate(cfgs):
        b.init(i, *start_fields(c, i))
    b.step(steps)
    st = b.stats()
    assert st["status"] == D.OK and not st["flags"].any()
    for i, c in enumerate(cfgs):
        ref = D.Lattice(c).init(*start_fields(c, i)).step(steps).fields()
        got = b.fields(i)
        for k in D.FIELD_NAMES:
            assert same(got[k], ref[k]), (bc, i, k)


def test_batch_instance_matches_oracle():
    c = CFGS[3]
    b = D.Batch([c]).set_run(steps_per_launch=50)
    f = start_fields(c, 3)
    b.init(0, *f).step(150)
    got = {k: np64(v) for k, v in b.fields(0).items()}
    wf, wg = c.rates()
    p = O.OracleParams(nx=c.nx, ny=c.ny, bc=c.bc, lam_override=wf, lam_phi_override=wg,
                       u_lid=c.u_lid, phi_lid=c.phi_lid, phi_wall=c.phi_wall)
    r32 = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)
    ref = O.OracleLattice(p).init(*[r32(a) for a in f]).step(150).fields()
    for k in ("ux", "uy", "phi"):
        err = math.sqrt(np.sum((got[k] - ref[k]) ** 2) / np.sum(ref[k] ** 2))
        assert err < 1e-5, (k, err)


@pytest.mark.parametrize("schedule", [0, 1])
def test_convergence_freezes_instance(schedule):
    """An instance whose residual drops below tol stops; its state is the one
    the single path reaches one step after the check that froze it."""
    slow = cfg(48, 48, "cavity", 0.2, check=20, u_lid=0.05)
    fast = cfg(48, 48, "cavity", 0.2, check=20, u_lid=0.05, phi_lid=0.7)
    ref = D.Lattice(slow).init(*start_fields(slow, 0))
    rs = []
    for _ in range(30):
        ref.step(20)
        rs.append(ref.stats()["residual"])
    tol = rs[10] * 1.0001
    first = next(k for k, r in enumerate(rs) if r < tol)   # checks at t = 20 (k + 1)
    t_tol = 20 * (first + 1)
    b = D.Batch([slow, fast]).set_run(tol=tol, steps_per_launch=40).set_schedule(schedule)
    b.init(0, *start_fields(slow, 0)).init(1, *start_fields(fast, 0))
    b.step(600)
    st = b.stats()
    assert st["flags"][0] == D.INST_CONVERGED and st["steps_to_tol"][0] == t_tol
    assert st["state_time"][0] == t_tol + 1
    frozen = b.fields(0)
    again = D.Lattice(slow).init(*start_fields(slow, 0)).step(t_tol + 1).fields()
    for k in D.FIELD_NAMES:
        assert same(frozen[k], again[k]), k
    # re-initialised later (the batch is at state time 600), the instance
    # counts its steps from that init
    b.init(0, *start_fields(slow, 0))
    b.step(600)
    st2 = b.stats()
    assert st2["init_time"][0] == 600
    assert st2["flags"][0] == D.INST_CONVERGED and st2["steps_to_tol"][0] == t_tol
    assert st2["state_time"][0] - st2["init_time"][0] == t_tol + 1


@pytest.mark.parametrize("schedule", [0, 1])
def test_instance_tolerance_and_step_limit(schedule):
    """Per-instance run settings: the same cavity three times in one batch,
    one frozen by its own tolerance, one by the batch's, one capped by its own
    step limit before it converges (flag INST_CAPPED, frozen at the first
    check at or past the limit).  The state each stops in is the single path's
    at the same time."""
    c = cfg(48, 48, "cavity", 0.2, check=20, u_lid=0.05)
    ref = D.Lattice(c).init(*start_fields(c, 0))
    rs = []
    for _ in range(30):
        ref.step(20)
        rs.append(ref.stats()["residual"])
    loose, tight = rs[5] * 1.0001, rs[20] * 1.0001
    t_loose = 20 * (next(k for k, r in enumerate(rs) if r < loose) + 1)
    t_tight = 20 * (next(k for k, r in enumerate(rs) if r < tight) + 1)
    b = D.Batch([c, c, c]).set_run(tol=tight, steps_per_launch=40).set_schedule(schedule)
    b.set_instance_run(0, tol=loose)
    b.set_instance_run(2, tol=1e-30, max_steps=170)     # limit between two checks
    for i in range(3):
        b.init(i, *start_fields(c, 0))
    b.step(800)
    st = b.stats()
    assert list(st["flags"]) == [D.INST_CONVERGED, D.INST_CONVERGED, D.INST_CAPPED]
    assert st["steps_to_tol"][0] == t_loose and st["steps_to_tol"][1] == t_tight
    assert st["steps_to_tol"][2] == -1 and st["state_time"][2] == 181   # check at t = 180
    capped = b.fields(2)
    again = D.Lattice(c).init(*start_fields(c, 0)).step(181).fields()
    for k in D.FIELD_NAMES:
        assert same(capped[k], again[k]), k
    # settings survive a re-init; a negative tolerance returns to the batch's
    b.set_instance_run(0, tol=-1.0)
    b.init(0, *start_fields(c, 0)).init(2, *start_fields(c, 0))
    b.step(800)
    st2 = b.stats()
    assert st2["flags"][0] == D.INST_CONVERGED and st2["steps_to_tol"][0] == t_tight
    assert st2["flags"][2] == D.INST_CAPPED


def test_divergence_is_isolated():
    """A NaN in one instance's initial fields flags that instance only."""
    c0, c1 = cfg(32, 32, "periodic", 0.01), cfg(40, 24, "cavity", 0.05, u_lid=0.1)
    bad = list(start_fields(c0, 0))
    bad[0] = bad[0].copy(); bad[0][5, 7] = np.nan
    b = D.Batch([c0, c1]).set_run(steps_per_launch=25)
    b.init(0, *bad).init(1, *start_fields(c1, 1)).step(50)
    st = b.stats()
    assert st["flags"][0] == D.INST_DIVERGED and st["flags"][1] == 0
    ref = D.Lattice(c1).init(*start_fields(c1, 1)).step(50).fields()
    got = b.fields(1)
    for k in D.FIELD_NAMES:
        assert same(got[k], ref[k]), k


def test_c4_batch_every_instance_vs_oracle():
    """The 512-cavity batch (sizes 64..512, Re log-uniform in [100, 3200],
    Pe = Re, seed 0) after 200 steps, tiles from the autotuner: every instance
    against the oracle (u, phi within 1e-5; S within 1e-5 of the largest
    component's RMS)."""
    draws = inputs.cavity_batch(512, seed=0)
    cfgs = []
    for d in draws:
        n, U = d["n"], 0.1
        w = rate(U * n / d["re"])
        wg = rate(U * n / d["pe"])
        cfgs.append(D.Config(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0,
                             omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                             omega_g=(0, wg, wg, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2), check_every=100))
    b = D.Batch(cfgs).set_run(tol=0.0, steps_per_launch=100)
    b.autotune(trial_steps=5, cache=False)
    for i, c in enumerate(cfgs):
        F = inputs.rest(c.nx, c.ny, phi=0.0)
        b.init(i, F.rho, F.ux, F.uy, F.phi)
    b.step(200)
    st = b.stats()
    assert st["status"] == D.OK
    worst = {"u": 0.0, "phi": 0.0, "S": 0.0}
    for i, d in enumerate(draws):
        c, n = cfgs[i], d["n"]
        wf, wg = c.rates()
        p = O.OracleParams(nx=n, ny=n, bc="cavity", lam_override=wf, lam_phi_override=wg,
                           u_lid=c.u_lid, phi_lid=1.0, phi_wall=0.0)
        F = inputs.rest(n, n, phi=0.0)
        ref = O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi).step(200).fields()
        got = {k: np64(v) for k, v in b.fields(i).items()}
        e_u = math.sqrt(np.sum((got["ux"] - ref["ux"]) ** 2 + (got["uy"] - ref["uy"]) ** 2) /
                        np.sum(ref["ux"] ** 2 + ref["uy"] ** 2))
        e_phi = math.sqrt(np.sum((got["phi"] - ref["phi"]) ** 2) / np.sum(ref["phi"] ** 2))
        srms = max(math.sqrt(np.mean(ref[k] ** 2)) for k in ("sxx", "sxy", "syy"))
        e_s = max(math.sqrt(np.mean((got[k] - ref[k]) ** 2)) for k in ("sxx", "sxy", "syy")) / srms
        assert e_u < 1e-5 and e_phi < 1e-5 and e_s < 1e-5, (i, n, e_u, e_phi, e_s)
        for k, v in (("u", e_u), ("phi", e_phi), ("S", e_s)):
            worst[k] = max(worst[k], v)
    print("512 instances after 200 steps, worst relative errors", worst)


def test_c4_long_run_small_instances_vs_oracle():
    """The batched-cavity recipe (seed 0, first 64 draws: all sizes mixed in one
    persistent launch) run for the full 20000 steps; the first 64^2, 96^2 and
    128^2 instances against the FP64 oracle: u, phi and S within 1e-5 or three
    times the error of the oracle's own FP32-storage emulation, omega likewise
    where |phi| > 2e-3 (phi = 0 on three walls)."""
    draws = inputs.cavity_batch(64, seed=0)
    cfgs = []
    for d in draws:
        n, U = d["n"], 0.1
        w, wg = rate(U * n / d["re"]), rate(U * n / d["pe"])
        cfgs.append(D.Config(nx=n, ny=n, bc="cavity", u_lid=U, phi_lid=1.0, phi_wall=0.0,
                             omega_f=(0, 0, 0, 1.2, w, w, 1.2, 1.2, 1.2),
                             omega_g=(0, wg, wg, 1.2, 1.2, 1.2, 1.2, 1.2, 1.2), check_every=100))
    b = D.Batch(cfgs).set_run(tol=0.0, steps_per_launch=1000)
    for i, c in enumerate(cfgs):
        F = inputs.rest(c.nx, c.ny, phi=0.0)
        b.init(i, F.rho, F.ux, F.uy, F.phi)
    steps = 20000
    b.step(steps)
    assert b.stats()["status"] == D.OK
    picks = {}
    for i, d in enumerate(draws):
        if d["n"] in (64, 96, 128):
            picks.setdefault(d["n"], i)
    assert len(picks) == 3, sorted(picks)

    def errs(got, ref, sel):
        e = {"u": math.sqrt(np.sum((got["ux"] - ref["ux"]) ** 2 + (got["uy"] - ref["uy"]) ** 2) /
                            np.sum(ref["ux"] ** 2 + ref["uy"] ** 2)),
             "phi": math.sqrt(np.sum((got["phi"] - ref["phi"]) ** 2) / np.sum(ref["phi"] ** 2))}
        srms = max(math.sqrt(np.mean(ref[k] ** 2)) for k in ("sxx", "sxy", "syy"))
        e["S"] = max(math.sqrt(np.mean((got[k] - ref[k]) ** 2)) for k in ("sxx", "sxy", "syy")) / srms
        e["omega"] = math.sqrt(np.sum((got["omega"][sel] - ref["omega"][sel]) ** 2) /
                               np.sum(ref["omega"][sel] ** 2))
        return e

    for n, i in sorted(picks.items()):
        c = cfgs[i]
        wf, wg = c.rates()
        F = inputs.rest(n, n, phi=0.0)
        out = []
        for storage in ("fp64", "fp32"):
            p = O.OracleParams(nx=n, ny=n, bc="cavity", lam_override=wf, lam_phi_override=wg,
                               u_lid=c.u_lid, phi_lid=1.0, phi_wall=0.0, storage=storage)
            out.append(O.OracleLattice(p).init(F.rho, F.ux, F.uy, F.phi).step(steps).fields())
        ref, emu = out
        sel = np.abs(ref["phi"]) > 2e-3
        got = {k: np64(v) for k, v in b.fields(i).items()}
        e, floor = errs(got, ref, sel), errs(emu, ref, sel)
        print(n, "errors", {k: f"{v:.2e}" for k, v in e.items()},
              "floor", {k: f"{v:.2e}" for k, v in floor.items()})
        for k, v in e.items():
            assert v <= max(1e-5, 3 * floor[k]), (n, k, v, floor[k])


def test_barrier_wait_runs_out_and_reports_timeout():
    """One CTA never arrives (a flag nothing sets): the others give up after the
    bounded wait, the launch ends, stats reports ETIMEOUT, and the context stays
    usable (a new batch runs correctly afterwards)."""
    c = cfg(64, 64, "periodic", 0.01)
    b = D.Batch([c]).set_run(steps_per_launch=5, barrier_timeout_s=0.3)
    b.init(0, *start_fields(c, 0)).debug_skip_barrier(0).step(5)
    st = b.stats()
    assert st["status"] == D.ETIMEOUT
    b.close()
    torch.cuda.synchronize()
    b2 = D.Batch([c]).set_run(steps_per_launch=5)
    b2.init(0, *start_fields(c, 0)).step(10)
    ref = D.Lattice(c).init(*start_fields(c, 0)).step(10).fields()
    assert same(b2.fields(0)["omega"], ref["omega"])

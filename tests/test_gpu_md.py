"""Velocity-Verlet NVE with the model's forces: total energy is conserved to
second order in the step, momentum stays zero (Newton's third law per
structure, Eq. 3), positions stay wrapped, and the forces returned by a step
are those of a fresh forward pass at the new positions."""
import numpy as np
import pytest
import torch

from paper_2507_00528_gb300 import gnep, md, synth

from gpu_common import rel_l2

pytestmark = pytest.mark.gpu

SHAPE = dict(n_max=(4, 4), basis=(8, 8), hidden=30, four_body=False)


def _model(batch):
    m = gnep.GNEP(**SHAPE, seed=101)
    m.compute_scale(m.neighbors(gnep.DeviceBatch.from_host(batch)))
    return m


def _run(dt, steps, batch, model):
    sim = md.NVE(model, batch, temperature=300.0, seed=3)
    e = [sim.total()]
    for _ in range(steps):
        sim.step(dt)
        e.append(sim.total())
    return sim, np.array(e)


def test_energy_conservation_scales_with_dt_squared():
    b = synth.make_batch([64, 40, 50], [0, 1, 2], np.random.default_rng(11))
    m = _model(b)
    n_atoms = b.sizes()
    _, e1 = _run(1.0, 200, b, m)
    _, e2 = _run(0.5, 400, b, m)
    fl1 = np.abs(e1 - e1[0]).max(0) / n_atoms  # eV / atom, per structure
    fl2 = np.abs(e2 - e2[0]).max(0) / n_atoms
    print("energy fluctuation per atom dt=1:", fl1, "dt=0.5:", fl2)
    assert fl1.max() < 2e-3
    # velocity Verlet: halving the step quarters the fluctuation (within FP32 force noise)
    assert np.all(fl2 < 0.45 * fl1 + 2e-6), (fl1, fl2)


def test_momentum_wrapping_and_forces_after_steps():
    b = synth.make_batch([48, 33], [1, 2], np.random.default_rng(12))
    m = _model(b)
    sim, _ = _run(1.0, 50, b, m)
    p = sim.momentum()
    v = sim.vel.cpu().numpy()
    ref = np.sqrt(sim.mass.mean() * np.mean(v * v)) * np.sqrt(b.n_atoms)
    assert np.abs(p).max() < 1e-4 * ref, p
    # positions wrapped into their cell
    pos = sim.pos.cpu().numpy()
    for s in range(b.n_struct):
        a0, a1 = b.struct_off[s], b.struct_off[s + 1]
        f = pos[a0:a1] @ np.linalg.inv(b.cell[s])
        assert f.min() > -1e-9 and f.max() < 1.0 + 1e-9
    # the step's forces equal a fresh forward pass at the new positions
    moved = synth.Batch(b.struct_off.copy(), pos, b.types.copy(), b.cell.copy())
    nl = m.neighbors(gnep.DeviceBatch.from_host(moved))
    _, Es, F, _ = m.forward(nl)
    assert rel_l2(sim.F.double().cpu().numpy(), F.double().cpu().numpy()) < 1e-6
    assert rel_l2(sim.E_pot.cpu().numpy(), Es.cpu().numpy()) < 1e-9


def test_rejects_host_arrays():
    b = synth.make_batch([20], [1], np.random.default_rng(13))
    m = _model(b)
    sim = md.NVE(m, b)
    sim.pos = sim.pos.cpu()
    with pytest.raises(gnep._lib.GnepError):
        sim.step(1.0)


def test_trajectory_matches_the_oracle_integrator():
    """Ten velocity-Verlet steps of gnep_md_verlet (FP32 forces, FP64 positions
    and velocities) against the oracle's FP64 velocity Verlet from the same
    start: positions, velocities, forces and potential energies after every
    step, within the FP32 force tolerance carried through the integrator."""
    import oracle as O
    b = synth.make_batch([24, 19], [0, 2], np.random.default_rng(14))
    cfg = O.Cfg(nq_r=5, nq_a=5, k_r=9, k_a=9, hidden=30)
    P = synth.uniform_params(cfg.n_params, 101)
    s = O.descriptor_scale(cfg, P.astype(np.float64), b).astype(np.float32)
    m = gnep.GNEP(**SHAPE)
    m.set_params(torch.from_numpy(P))
    m.set_scale(torch.from_numpy(s))
    sim = md.NVE(m, b, temperature=600.0, seed=5)
    v0 = sim.vel.cpu().numpy().copy()
    traj = O.md_verlet(cfg, P.astype(np.float64), s.astype(np.float64), b, v0, 1.0 / sim.mass, 1.0, 10)
    for k in range(10):
        sim.step(1.0)
        x, v, F, Es = traj[k]
        d = sim.pos.cpu().numpy() - x
        for st in range(b.n_struct):  # minimum image
            a0, a1 = b.struct_off[st], b.struct_off[st + 1]
            f = d[a0:a1] @ np.linalg.inv(b.cell[st])
            d[a0:a1] = (f - np.round(f)) @ b.cell[st]
        assert np.abs(d).max() < 1e-7, (k, np.abs(d).max())
        assert np.abs(sim.vel.cpu().numpy() - v).max() < 1e-8 + 1e-6 * np.abs(v).max()
        assert rel_l2(sim.F.double().cpu().numpy(), F) < 1e-5
        assert rel_l2(sim.E_pot.cpu().numpy(), Es) < 1e-6

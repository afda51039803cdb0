"""Batched cavities and the request loop, through the C ABI, against single
runs and the FP64 oracle.

* a batch of uneven meshes advances each cavity exactly as the oracle does
  (FP64 <= 1e-12 per step, FP32 <= 1e-5);
* each cavity's result is the same alone (batch of one) and in a mix of
  others, within the same tolerances;
* per-slot run control: tolerance and step caps stop slots independently,
  slots are reused after removal;
* the request loop retires requests with the Nusselt numbers a single run
  of the same request gives.
"""
import numpy as np
import pytest

from paper_2202_13449_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

TOL = {capi.FP64: 1e-12, capi.FP32: 1e-5}


def rel(a, b, floor):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(float(np.max(np.abs(b))), floor))


SPECS = [  # (nx, ny, phi, Ra, seed)
    (37, 21, 1.5, 1e5, 1),
    (64, 64, 0.0, 1e3, 2),
    (29, 45, 2.2, 3e4, 3),
    (96, 33, 1.0, 1e6, 4),
]


def mesh(orc, nx, ny, phi):
    return orc.tanh_faces(nx, float(nx), phi), orc.tanh_faces(ny, float(nx) * ny / nx, phi)


def add(b, orc, spec, state):
    nx, ny, phi, Ra, _ = spec
    xf, yf = mesh(orc, nx, ny, phi)
    dt = 0.5 * float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
    s = b.add(xf, yf, Ra, 0.71, 0.1, dt)
    b.set_state(s, *state)
    return s, xf, yf, dt


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_batch_matches_oracle_per_cavity(orc, precision):
    b = capi.Batch(precision, 8)
    slots = []
    for spec in SPECS:
        st = inputs.perturbed_state(spec[0], spec[1], seed=spec[4])
        s, xf, yf, dt = add(b, orc, spec, st)
        b.arm(s, 0.0, 12)
        slots.append((s, xf, yf, dt, st, spec))
    b.step(12)
    status, steps, _ = b.poll()
    for s, xf, yf, dt, st, spec in slots:
        assert status[s] == capi.SLOT_MAX_STEPS and steps[s] == 12
        nu, chi, bg = orc.params_from_ra(spec[3], 0.71, 0.1, float(spec[0]))
        p = orc.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=bg, dt=dt)
        ref, _, rc = orc.step(p, st, 12)
        got = b.get_state(s)
        for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
            assert rel(got[q], ref[q], floor) < 10 * TOL[precision], (spec, q)
    b.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_same_result_alone_and_in_the_mix(orc, precision):
    """The first cavity stepped alone and stepped together with three others
    (which changes the work list and the chunking of the marching kernel)."""
    spec = SPECS[0]
    st = inputs.perturbed_state(spec[0], spec[1], seed=11)
    alone = capi.Batch(precision, 1)
    s0, *_ = add(alone, orc, spec, st)
    alone.arm(s0, 0.0, 40)
    alone.step(40)
    a = alone.get_state(s0)
    alone.close()
    mix = capi.Batch(precision, 8)
    sm = None
    for k, sp in enumerate(SPECS):
        stk = st if k == 0 else inputs.perturbed_state(sp[0], sp[1], seed=20 + k)
        s, *_ = add(mix, orc, sp, stk)
        mix.arm(s, 0.0, 40)
        if k == 0:
            sm = s
    mix.step(40)
    m = mix.get_state(sm)
    mix.close()
    for q, floor in ((1, 1e-2), (2, 1e-2), (3, 1.0)):
        assert rel(m[q], a[q], floor) < TOL[precision], q


def test_slots_stop_independently_and_are_reused(orc):
    b = capi.Batch(capi.FP64, 3)
    ids = []
    for k, spec in enumerate(SPECS[:3]):
        st = inputs.conduction_state(*mesh(orc, spec[0], spec[1], spec[2]))
        s, *_ = add(b, orc, spec, st)
        ids.append(s)
    b.arm(ids[0], 0.0, 5)
    b.arm(ids[1], 0.0, 50)
    b.arm(ids[2], 1e-30, 30)
    b.step(60)
    status, steps, res = b.poll()
    assert steps[ids[0]] == 5 and steps[ids[1]] == 50 and steps[ids[2]] == 30
    assert status[ids[0]] == capi.SLOT_MAX_STEPS
    b.remove(ids[1])
    status, _, _ = b.poll()
    assert status[ids[1]] == capi.SLOT_EMPTY
    spec = SPECS[3]
    st = inputs.conduction_state(*mesh(orc, spec[0], spec[1], spec[2]))
    s, *_ = add(b, orc, spec, st)
    assert s == ids[1]
    b.arm(s, 0.0, 7)
    b.step(7)
    _, steps, _ = b.poll()
    assert steps[s] == 7 and steps[ids[0]] == 5
    b.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_request_loop_results_equal_single_runs(orc, precision):
    reqs = [(0.002 * k, n, Ra, Pr) for k, (n, Ra, Pr) in enumerate(
        [(16, 1e3, 0.71), (24, 3e3, 7.0), (20, 1e4, 0.71), (16, 2e3, 7.0), (32, 1e3, 0.71),
         (18, 5e3, 0.71)])]
    tol, cap = 1e-6, 30000
    res, el = capi.serve(reqs, max_slots=4, tol=tol, max_steps=cap, chunk_steps=64,
                         precision=precision, time_limit_s=120.0)
    for (t, n, Ra, Pr), r in zip(reqs, res):
        assert r["status"] in (capi.SLOT_CONVERGED, capi.SLOT_MAX_STEPS)
        assert r["t_admit"] >= t and r["t_finish"] >= r["t_admit"]
        xf = inputs.uniform_faces(n)
        s = capi.Solver(xf, xf, precision)
        s.set_params(Ra, Pr, 0.1, 0.0)
        rc, steps, _ = s.run_to_steady(tol, cap)
        assert abs(steps - r["steps"]) <= 1, (steps, r["steps"])
        tol_nu = 1e-10 if precision == capi.FP64 else 1e-4
        for which, key in ((capi.NU_WEST, "nu_hot"), (capi.NU_EAST, "nu_cold")):
            want = s.nusselt(which)
            if steps == r["steps"]:
                assert abs(r[key] - want) <= tol_nu * abs(want), (n, Ra, key, r[key], want)
        s.close()


def test_batch_workload_stays_stable_with_the_automatic_step():
    """The seeded batch workload (sides 32..256, tanh phi 1..2.5, Ra 1e3..1e6)
    with dt = 0 (the stability rule): no cavity diverges in 300 steps."""
    specs = inputs.batch_specs(96, 1234)
    b = capi.Batch(capi.FP32, len(specs))
    for sp in specs:
        xf = capi.tanh_faces(sp.n, float(sp.n), sp.phi)
        s = b.add(xf, xf, sp.Ra, sp.Pr, 0.1, 0.0)
        b.arm(s, 0.0, 300)
    b.step(300)
    status, steps, _ = b.poll()
    assert all(st == capi.SLOT_MAX_STEPS for st in status[:len(specs)]), status
    assert all(k == 300 for k in steps[:len(specs)])
    b.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_batch_raw_checkpoint_resumes_bit_for_bit(precision):
    """Every slot's records taken after some batched steps and restored into
    a fresh batch continue bit for bit like the uninterrupted batch."""
    def build():
        b = capi.Batch(precision, 8)
        slots = []
        for nx, ny, phi, Ra, seed in SPECS:
            xf = capi.tanh_faces(nx, float(nx), phi)
            yf = capi.tanh_faces(ny, float(nx) * ny / nx, phi)
            dt = 0.5 * float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
            s = b.add(xf, yf, Ra, 0.71, 0.1, dt)
            b.set_state(s, *inputs.perturbed_state(nx, ny, seed=seed))
            slots.append(s)
        return b, slots

    a, sa = build()
    for s in sa:
        a.arm(s, 0.0, 20)
    a.step(20)
    recs = [a.get_state_raw(s) for s in sa]
    for s, (r, _) in zip(sa, recs):
        rec_bytes = 16 if precision == capi.FP32 else 32
        nx, ny = SPECS[sa.index(s)][0], SPECS[sa.index(s)][1]
        assert r.size == a.raw_bytes(s) == nx * ny * rec_bytes
    for s in sa:
        a.arm(s, 0.0, 15)
    a.step(15)
    want = [a.get_state(s) for s in sa]
    b, sb = build()
    for s, (r, tu) in zip(sb, recs):
        b.set_state_raw(s, r, tu)
        b.arm(s, 0.0, 15)
    b.step(15)
    for s_a, s_b, wv in zip(sa, sb, want):
        got = b.get_state(s_b)
        for q in range(4):
            np.testing.assert_array_equal(got[q], wv[q])
        np.testing.assert_array_equal(b.get_state_raw(s_b)[0], a.get_state_raw(s_a)[0])
    with pytest.raises(capi.RTLBFSError):
        b.set_state_raw(sb[0], recs[0][0], 3.0)  # not a power of two
    with pytest.raises(ValueError):
        b.set_state_raw(sb[0], recs[0][0][:-16], recs[0][1])
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_batch_records_of_many_slots_in_one_call(precision):
    """rtlbfs_batch_get/set_states_raw equal the per-slot calls byte for
    byte, and refuse bad arguments before copying anything."""
    b = capi.Batch(precision, 8)
    slots = []
    for nx, ny, phi, Ra, seed in SPECS:
        xf = capi.tanh_faces(nx, float(nx), phi)
        yf = capi.tanh_faces(ny, float(nx) * ny / nx, phi)
        s = b.add(xf, yf, Ra, 0.71, 0.1, 0.0)
        b.set_state(s, *inputs.perturbed_state(nx, ny, seed=seed))
        b.arm(s, 0.0, 7)
        slots.append(s)
    b.step(7)
    one = [b.get_state_raw(s) for s in slots]
    outs = [np.zeros(b.raw_bytes(s), dtype=np.uint8) for s in slots]
    tu = b.get_states_raw(slots, outs)
    for (r, t), o, u in zip(one, outs, tu):
        np.testing.assert_array_equal(o, r)
        assert u == t
    # set many: scramble every slot, restore all in one call, read back
    for s in slots:
        b.set_state(s, *inputs.perturbed_state(*reversed(b.shapes[s]), seed=99))
    b.set_states_raw(slots, outs, tu)
    for s, (r, _) in zip(slots, one):
        np.testing.assert_array_equal(b.get_state_raw(s)[0], r)
    # a slot not in use, or a bad unit: nothing copied
    before = [b.get_state_raw(s)[0].copy() for s in slots]
    with pytest.raises(capi.RTLBFSError):
        b.set_states_raw(slots[:1] + [7], [outs[0], outs[0]], [tu[0], tu[0]])
    with pytest.raises(capi.RTLBFSError):
        b.set_states_raw(slots, outs, [3.0] * len(slots))
    for s, r in zip(slots, before):
        np.testing.assert_array_equal(b.get_state_raw(s)[0], r)
    b.close()


def test_batch_arm_many_equals_arming_each_slot():
    """One arm_many launch leaves every slot armed as rtlbfs_batch_arm does:
    the same stop step and the same fields; a bad slot arms none."""
    def build():
        b = capi.Batch(capi.FP32, 8)
        slots = []
        for nx, ny, phi, Ra, seed in SPECS:
            xf = capi.tanh_faces(nx, float(nx), phi)
            yf = capi.tanh_faces(ny, float(nx) * ny / nx, phi)
            s = b.add(xf, yf, Ra, 0.71, 0.1, 0.0)
            b.set_state(s, *inputs.perturbed_state(nx, ny, seed=seed))
            slots.append(s)
        return b, slots

    a, sa = build()
    for s in sa:
        a.arm(s, 0.0, 9)
    a.step(12)
    m, sm = build()
    with pytest.raises(capi.RTLBFSError):
        m.arm_many(sm + [7], 0.0, 9)
    m.step(3)  # nothing armed: no slot moves
    st0, steps0, _ = m.poll()
    assert all(steps0[s] == 0 for s in sm)
    m.arm_many(sm, 0.0, 9)
    m.step(12)
    st_a, steps_a, _ = a.poll()
    st_m, steps_m, _ = m.poll()
    for s_a, s_m in zip(sa, sm):
        assert steps_m[s_m] == steps_a[s_a] == 9
        assert st_m[s_m] == st_a[s_a] == capi.SLOT_MAX_STEPS
        for q in range(4):
            np.testing.assert_array_equal(m.get_state(s_m)[q], a.get_state(s_a)[q])
    a.close()
    m.close()


def test_batch_schedule_is_settable():
    """rtlbfs_batch_set_schedule: the tile kernel and the marching kernel
    advance a batch to the same fields (FP64: the same arithmetic up to the
    order of a few sums); the persistent kernel is refused for a batch."""
    out = []
    for kernel, rows in ((0, 32), (1, 8)):
        b = capi.Batch(capi.FP64, 8)
        slots = []
        for nx, ny, phi, Ra, seed in SPECS:
            xf = capi.tanh_faces(nx, float(nx), phi)
            yf = capi.tanh_faces(ny, float(nx) * ny / nx, phi)
            s = b.add(xf, yf, Ra, 0.71, 0.1, 0.0)
            b.set_state(s, *inputs.perturbed_state(nx, ny, seed=seed))
            b.arm(s, 0.0, 10)
            slots.append(s)
        b.set_schedule(kernel, rows)
        with pytest.raises(capi.RTLBFSError):
            b.set_schedule(2, 0)
        b.step(10)
        out.append([b.get_state(s) for s in slots])
        b.close()
    for sa, sb in zip(*out):
        for q in range(4):
            assert rel(sb[q], sa[q], 1e-3) < 1e-12

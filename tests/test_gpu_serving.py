"""Serving engine: continuous batching of many drones' control steps (GPU).

The bar: every drone's results are the same alone and in the mix (bit-identical:
each drone's warm start and Philox counter live on the device, and every kernel
reduces in a fixed order), also when a small device-memory budget forces its
context to be evicted to host memory and restored between requests.  Both
engines are held to it: batched launches (every admissible request of a window
in one set of launches) and one captured step graph per drone.  Across the two
engines (and against mppi_step) the results agree within the FP32 control bar
of the parity tests, 1e-4: the batched kernels run the same device functions on
the same data, but they are separately compiled kernels, whose floating-point
contractions may differ (1 ulp has been seen).
"""
CTRL_ATOL = 1e-4
import time

import numpy as np
import pytest

import workloads as W
from paper_2603_07199_gb300 import binding as B

from .gpu_helpers import flat_layers, make_config

pytestmark = pytest.mark.gpu


MODES = {"bf16": B.MPPI_SDF_MLP_BF16, "fp16": B.MPPI_SDF_MLP_FP16, "fp8": B.MPPI_SDF_MLP_FP8,
         "fp32": B.MPPI_SDF_MLP_FP32, "analytic": B.MPPI_SDF_ANALYTIC}


def _drone_cfg(d, mode="bf16"):
    return make_config(d["params"], mode, d["G"])


def _run(fleet, requests, budget=0, max_inflight=16, mode="bf16", layers=None, batching=1, single_cta=None):
    """Submit (drone index, state) requests in order without waiting; return controls per request."""
    cfg = B.mppi_server_config_default()
    cfg.hbm_budget_bytes = budget
    cfg.max_inflight = max_inflight
    cfg.sdf_mode = MODES[mode]
    cfg.batching = batching
    if single_cta is not None:
        cfg.sdf_single_cta = single_cta
    srv = B.mppi_server_create(cfg)
    keep = flat_layers(layers) if layers is not None else None
    if keep is not None:
        B.mppi_server_set_sdf_weights(srv, keep)
    tickets = []
    for di, state in requests:
        d = fleet[di]
        tickets.append((di, B.mppi_server_submit(srv, d["drone_id"], _drone_cfg(d, mode), np.ascontiguousarray(state, np.float32),
                                                 d["G"], np.ascontiguousarray(d["poses"]), np.ascontiguousarray(d["latents"]))))
    outs, lats = [None] * len(tickets), [0.0] * len(tickets)
    t0 = time.time()
    pending = set(range(len(tickets)))
    while pending and time.time() - t0 < 120:
        for i in list(pending):
            di, t = tickets[i]
            U = np.zeros((fleet[di]["params"]["H"], 4), np.float32)
            st, lat = B.mppi_server_poll(srv, t, U)
            if st == B.MPPI_OK:
                outs[i], lats[i] = U, lat
                pending.discard(i)
        time.sleep(0.0005)
    stats = B.mppi_server_get_stats(srv)
    B.mppi_server_destroy(srv)
    assert not pending, "requests did not finish"
    return outs, lats, stats


def _states(fleet, n_steps, seed=7):
    rng = np.random.default_rng(seed)
    return {i: [np.asarray(d["state"], np.float32) + np.float32(0.05) * rng.standard_normal(13).astype(np.float32) * np.array(
        [1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 1], np.float32) for _ in range(n_steps)] for i, d in enumerate(fleet)}


@pytest.mark.parametrize("batching", [1, 0])
def test_results_are_the_same_alone_and_in_the_mix(lib, batching):
    fleet = W.serving_fleet(8, seed=4, Ks=(256, 512, 1024), Hs=(10, 20, 30))
    layers = W.xavier_mlp(1)
    n_steps = 4
    states = _states(fleet, n_steps)
    target = 3
    alone, _, _ = _run(fleet, [(target, states[target][s]) for s in range(n_steps)], layers=layers, batching=batching)
    mix_reqs = [(i, states[i][s]) for s in range(n_steps) for i in range(len(fleet))]
    mix, lats, stats = _run(fleet, mix_reqs, layers=layers, batching=batching)
    got = [mix[j] for j, (i, _) in enumerate(mix_reqs) if i == target]
    for a, b in zip(alone, got):
        np.testing.assert_array_equal(a, b)
    assert stats["completed"] == len(mix_reqs) and stats["evictions"] == 0
    assert all(l > 0 for l in lats)
    if batching:
        assert stats["batches"] > 0


def _mixed_fleet():
    """Drones that take every rollout form: a warp per rollout (H > 32, K < 8192), half warps with
    two and four steps per lane (H <= 32; K >= 8192), and the rotor-thrust-rate model."""
    fleet = W.serving_fleet(4, seed=21, Ks=(300,), Hs=(50,))
    fleet[1]["params"] = dict(fleet[1]["params"], K=256, H=10)
    fleet[2]["params"] = dict(fleet[2]["params"], K=8192, H=40)
    rot = fleet[3]
    rot["params"] = dict(W.rotor_params(512, 20), seed=rot["params"]["seed"], drone_id=rot["params"]["drone_id"])
    rot["state"] = W.rotor_state([0.2, -0.1, 0.3])
    return fleet


@pytest.mark.parametrize("batching", [1, 0])
@pytest.mark.parametrize("mode", ["fp16", "bf16"])
def test_sdf_kernel_forms_give_the_same_results(lib, mode, batching):
    """The server's default single-CTA SDF kernels and the CTA-pair form (batched: every drone's
    tiles padded to an even count, so a pair's two tiles belong to one drone) give every drone
    bit-identical controls, for a fleet whose drones have odd and even tile counts."""
    fleet = _mixed_fleet()
    fleet[0]["params"] = dict(fleet[0]["params"], H=43)          # 101 tiles
    layers = W.xavier_mlp(1)
    assert len({(d["params"]["K"] * d["params"]["H"] + 127) // 128 % 2 for d in fleet}) == 2
    n_steps = 2
    rng = np.random.default_rng(23)
    states = {i: [np.asarray(d["state"], np.float32) + np.float32(0.05) * rng.standard_normal(len(d["state"])).astype(
        np.float32) * (np.arange(len(d["state"])) < 6) for _ in range(n_steps)] for i, d in enumerate(fleet)}
    reqs = [(i, states[i][s]) for s in range(n_steps) for i in range(len(fleet))]
    single, _, _ = _run(fleet, reqs, mode=mode, layers=layers, batching=batching)
    pair, _, _ = _run(fleet, reqs, mode=mode, layers=layers, batching=batching, single_cta=0)
    for a, b in zip(single, pair):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", ["fp16", "bf16", "fp8", "fp32", "analytic"])
def test_batched_engine_equals_per_drone_engine(lib, mode):
    """The batched launches give every drone the results of its own step graph (within the FP32
    control bar) in every SDF mode (FP32 runs its SDF kernel per drone inside the batch) and for
    every rollout form."""
    fleet = _mixed_fleet()
    layers = W.xavier_mlp(1)
    n_steps = 3
    rng = np.random.default_rng(22)
    states = {i: [np.asarray(d["state"], np.float32) + np.float32(0.05) * rng.standard_normal(len(d["state"])).astype(
        np.float32) * (np.arange(len(d["state"])) < 6) for _ in range(n_steps)] for i, d in enumerate(fleet)}
    reqs = [(i, states[i][s]) for s in range(n_steps) for i in range(len(fleet))]
    batched, _, st_b = _run(fleet, reqs, mode=mode, layers=layers, batching=1)
    per_drone, _, _ = _run(fleet, reqs, mode=mode, layers=layers, batching=0)
    worst = max(float(np.max(np.abs(a - b))) for a, b in zip(batched, per_drone))
    print(f"{mode}: largest control difference batched vs per-drone graphs {worst:.3e}")
    assert worst <= CTRL_ATOL
    assert st_b["batches"] > 0


def test_batched_engine_shares_launches(lib):
    """After one warm-up request per drone (which creates the drones' contexts), 32 drones' next
    requests submitted back to back cannot all get a batch of their own (four batches run at
    once): several drones' steps share launches, with the per-drone engine's results."""
    fleet = W.serving_fleet(32, seed=31, Ks=(256, 512), Hs=(10, 20))
    layers = W.xavier_mlp(1)
    states = _states(fleet, 3, seed=32)
    reqs = [(i, states[i][s]) for s in range(3) for i in range(len(fleet))]
    results = {}
    for batching in (1, 0):
        cfg = B.mppi_server_config_default()
        cfg.max_inflight = 64
        cfg.sdf_mode = MODES["fp16"]
        cfg.batching = batching
        srv = B.mppi_server_create(cfg)
        B.mppi_server_set_sdf_weights(srv, flat_layers(layers))
        outs, b0 = [], 0
        for n_phase, phase in enumerate((reqs[:32], reqs[32:])):
            if n_phase == 1:                  # contexts exist: count the batches of the second phase
                b0 = B.mppi_server_get_stats(srv)["batches"]
            tickets = [B.mppi_server_submit(srv, fleet[i]["drone_id"], _drone_cfg(fleet[i], "fp16"),
                                            np.ascontiguousarray(st, np.float32), fleet[i]["G"],
                                            np.ascontiguousarray(fleet[i]["poses"]),
                                            np.ascontiguousarray(fleet[i]["latents"])) for i, st in phase]
            for (i, _), t in zip(phase, tickets):
                U = np.zeros((fleet[i]["params"]["H"], 4), np.float32)
                t0 = time.time()
                while B.mppi_server_poll(srv, t, U)[0] != B.MPPI_OK:
                    assert time.time() - t0 < 60, "request did not finish"
                    time.sleep(0.0002)
                outs.append(U)
        batches = B.mppi_server_get_stats(srv)["batches"] - b0
        B.mppi_server_destroy(srv)
        results[batching] = (outs, batches)
    assert 0 < results[1][1] < len(reqs) - 32
    for a, b in zip(results[1][0], results[0][0]):
        np.testing.assert_allclose(a, b, atol=CTRL_ATOL, rtol=0)


def test_small_budget_evicts_and_restores_without_changing_results(lib):
    fleet = W.serving_fleet(4, seed=9, Ks=(512,), Hs=(20,))
    layers = W.xavier_mlp(1)
    n_steps = 3
    states = _states(fleet, n_steps, seed=8)
    reqs = [(i, states[i][s]) for s in range(n_steps) for i in range(len(fleet))]
    free, _, st_free = _run(fleet, reqs, layers=layers)
    one = st_free["peak_device_bytes"] // len(fleet)
    tight, _, st_tight = _run(fleet, reqs, budget=int(2.5 * one), max_inflight=2, layers=layers)
    assert st_tight["evictions"] > 0 and st_tight["restores"] > 0
    assert st_tight["peak_device_bytes"] <= int(2.5 * one)
    for a, b in zip(free, tight):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("batching", [1, 0])
def test_serving_matches_a_plain_context(lib, batching):
    """One drone through the server equals the same steps through mppi_step."""
    fleet = W.serving_fleet(1, seed=11, Ks=(700,), Hs=(12,))
    layers = W.xavier_mlp(1)
    d = fleet[0]
    states = _states(fleet, 3, seed=12)[0]
    served, _, _ = _run(fleet, [(0, s) for s in states], layers=layers, batching=batching)
    ctx = B.mppi_create(_drone_cfg(d))
    keep = flat_layers(layers)
    B.mppi_set_sdf_weights(ctx, keep)
    B.mppi_set_gates(ctx, d["G"], np.ascontiguousarray(d["poses"]), np.ascontiguousarray(d["latents"]))
    for s, u in zip(states, served):
        U = np.zeros((12, 4), np.float32)
        B.mppi_step(ctx, np.ascontiguousarray(s, np.float32), None, None, None, U)
        if batching:
            np.testing.assert_allclose(U, u, atol=CTRL_ATOL, rtol=0)
        else:
            np.testing.assert_array_equal(U, u)      # the same captured step graph
    B.mppi_destroy(ctx)


def test_serving_errors(lib):
    fleet = W.serving_fleet(1, seed=13, Ks=(256,), Hs=(10,))
    d = fleet[0]
    cfg = B.mppi_server_config_default()
    cfg.sdf_mode = B.MPPI_SDF_ANALYTIC
    cfg.hbm_budget_bytes = 1024          # smaller than any context
    srv = B.mppi_server_create(cfg)
    dc = _drone_cfg(d, "analytic")
    with pytest.raises(B.MppiError):
        B.mppi_server_submit(srv, 0, dc, np.ascontiguousarray(d["state"]), dc.max_gates + 1,
                             np.zeros((dc.max_gates + 1, 7), np.float32), None)
    t = B.mppi_server_submit(srv, 0, dc, np.ascontiguousarray(d["state"]), d["G"], np.ascontiguousarray(d["poses"]), None)
    U = np.zeros((10, 4), np.float32)
    t0 = time.time()
    with pytest.raises(B.MppiError) as e:
        while time.time() - t0 < 30:
            st, _ = B.mppi_server_poll(srv, t, U)
            time.sleep(0.001)
    assert e.value.code == B.MPPI_E_ADMISSION
    with pytest.raises(B.MppiError):
        B.mppi_server_poll(srv, 10 ** 9, U)
    B.mppi_server_destroy(srv)

"""Several plans in one launch per wave (idg_grid_many / idg_degrid_many,
the serving loop's shared work queue): every plan's grid and predicted
visibilities equal what idg_grid / idg_degrid give it alone (up to the order
of FP64 atomic adds), for plans of different sizes, batch counts, A-term
intervals and w layers; mismatched plans are refused."""
import os

import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu


def _plans(idg_mod, specs):
    import torch
    out = []
    for k, (n_st, n_t, n_ch, flags, scratch) in enumerate(specs):
        obs = synth.config(2, seed=20 + k, n_stations=n_st, n_timesteps=n_t, n_channels=n_ch)
        if flags & idg_mod.IDG_W_LAYERS:
            rng = np.random.default_rng(k)
            enu = obs.enu.copy()
            enu[:, 2] = rng.normal(0.0, 300.0, enu.shape[0])
            obs = synth.make_observation(enu, n_t, 2.0, obs.freqs, 4, obs.grid_size, obs.subgrid_size,
                                         obs.kernel_padding, obs.image_size, name="layers")
        rng = np.random.default_rng(100 + k)
        A = torch.as_tensor(synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)).cuda()
        vis = torch.as_tensor(synth.random_visibilities(rng, obs)).cuda()
        if scratch:
            os.environ["IDG_SCRATCH_BYTES"] = str(scratch)
        try:
            plan = idg_mod.Plan(obs, flags=flags)
        finally:
            os.environ.pop("IDG_SCRATCH_BYTES", None)
        out.append((obs, plan, A, vis))
    return out


def test_grid_and_degrid_many_equal_single_plan_calls(idg_mod, cuda_device):
    import torch
    per_sg = 4 * 96 * 96 * 8
    specs = [(6, 8, 12, 0, 0), (10, 12, 17, 0, 5 * per_sg), (4, 3, 5, 0, 0), (8, 12, 16, idg_mod.IDG_W_LAYERS, 0)]
    items = _plans(idg_mod, specs)
    assert items[1][1].stats().n_batches > 1 and items[3][1].stats().n_w_layers >= 2
    plans = [p for _, p, _, _ in items]
    A = [a for _, _, a, _ in items]
    vis = [v for _, _, _, v in items]
    grids = [torch.zeros(p.grid_shape(), dtype=torch.complex128, device="cuda") for p in plans]
    idg_mod.grid_many(plans, vis, A, grids)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    models, outs = [], []
    for (obs, plan, a, v), G in zip(items, grids):
        ref = torch.zeros_like(G)
        plan.grid(v, a, ref)
        plan.synchronize()
        err = float(torch.linalg.vector_norm(G - ref) / torch.linalg.vector_norm(ref))
        assert err < 1e-12, err
        M = torch.as_tensor((rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape)) * 1e-3).cuda()
        models.append(M)
        outs.append(torch.full_like(v, 7.0 + 7.0j))
    idg_mod.degrid_many(plans, models, A, outs)
    torch.cuda.synchronize()
    for (obs, plan, a, v), M, V in zip(items, models, outs):
        ref = torch.empty_like(v)
        plan.degrid(M, a, ref)
        plan.synchronize()
        # the same kernels; only the order of the shared-memory adds of the warps' partial sums differs
        d = (V - ref).abs().max().item() / ref.abs().max().item()
        assert d < 1e-6, d
    for p in plans:
        p.close()


def test_many_refuses_mismatched_plans(idg_mod, cuda_device):
    import torch
    a = synth.config(1, seed=1, n_stations=6)
    b = synth.config(2, seed=1, n_stations=6, n_timesteps=4)
    pa, pb = idg_mod.Plan(a), idg_mod.Plan(b)
    try:
        A = [torch.as_tensor(synth.aterms_identity(o.n_intervals, o.n_stations)).cuda() for o in (a, b)]
        V = [torch.zeros((o.n_baselines, o.n_timesteps, o.n_channels, 4), dtype=torch.complex64, device="cuda")
             for o in (a, b)]
        G = [torch.zeros((4, o.grid_size, o.grid_size), dtype=torch.complex128, device="cuda") for o in (a, b)]
        with pytest.raises(idg_mod.IdgError) as e:   # L = 32 and L = 96
            idg_mod.grid_many([pa, pb], V, A, G)
        assert e.value.status == 1
        with pytest.raises(idg_mod.IdgError) as e:   # the same plan twice
            idg_mod.grid_many([pa, pa], [V[0], V[0]], [A[0], A[0]], [G[0], G[0]])
        assert e.value.status == 1
    finally:
        pa.close()
        pb.close()

"""Split z-chunks of the two-step TV launches (option tv_split). On a shape
whose equal z-chunks leave the last wave of CTAs partly idle, the last tiles
are cut into shorter z-chunks and launched after the others. The prox does
not depend on the chunking: the same volume bit for bit with and without the
split, and the oracle's on a crop through the split tiles. A FISTA solve
(whose fused-final launch sums the restart product over its CTAs) and a
batched solve of the same hologram agree with it."""

import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Batch, Rihv, rihv_tv_split_plan

pytestmark = pytest.mark.gpu

NX, NY, NZ = 256, 1024, 32          # 8.4 M voxels: both kinds of launch split
OPT = dict(nx=NX, ny=NY, nz=NZ, wavelength=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6)


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def handle(**opts):
    h = Rihv(NX, NY, NZ, OPT["wavelength"], OPT["pitch"], OPT["z0"], OPT["dz"])
    if opts:
        h.set_options(**opts)
    return h


def volume(seed):
    return torch.from_numpy(synth.random_complex(synth.Stream(seed), (NZ, NY, NX))
                            .astype(np.complex64)).cuda()


def test_the_schedule_splits_on_this_shape():
    h = handle()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for final in (False, True):
        zc, split, zc2 = h.tv_schedule(final)
        assert 0 < zc2 < zc and 0 < split, (final, zc, split, zc2)
        assert (split, zc2) == rihv_tv_split_plan(NX, NY, NZ, final, zc, sms)
    h.set_options(tv_split=0)
    assert h.tv_schedule(False)[2] == 0 and h.tv_schedule(True)[2] == 0
    h.close()


@pytest.mark.parametrize("dims,k", [(3, 20), (3, 7), (2, 6)])
def test_prox_with_and_without_split(dims, k):
    v = volume(500 + k)
    outs = []
    for split in (1, 0):
        h = handle(tv_dims=dims, tv_split=split)
        out = torch.empty_like(v)
        h.prox_fused_lasso(v, 0.3, 0.05, k, out)
        torch.cuda.synchronize()
        outs.append(out)
        h.close()
    assert torch.equal(outs[0], outs[1])


def test_split_prox_matches_oracle_on_a_crop():
    """The crop covers the last tile rows (the tiles cut into shorter
    z-chunks) and every plane; its interior lies more than 5 voxels from the
    crop faces that are inside the volume (4 dual steps reach 4)."""
    v = volume(510)
    h = handle(tv_dims=3)
    out = torch.empty_like(v)
    h.prox_fused_lasso(v, 0.3, 0.05, 4, out)
    torch.cuda.synchronize()
    y0, x1, m = NY - 48, 64, 6
    crop = v[:, y0:, :x1].cpu().numpy().astype(np.complex128)
    ref = O.prox_fused_lasso(crop, 0.3, 0.05, 4, 3)
    got = out[:, y0:, :x1].cpu().numpy()
    inner = (slice(None), slice(m, None), slice(0, x1 - m))
    assert rel_l2(got[inner], ref[inner]) <= 1e-5
    h.close()


def test_solve_and_batch_with_split():
    op = O.Optics(**OPT)
    a = np.zeros(op.shape)
    st = synth.Stream(520)
    for _ in range(40):
        z, y, x = int(st.uniform(1)[0] * NZ), int(st.uniform(1)[0] * (NY - 4)), int(st.uniform(1)[0] * (NX - 4))
        a[z, y:y + 3, x:x + 3] = 1.0
    b = synth.intensity_hologram(O.forward(a, op), 0.01, synth.Stream(521).normal(NX * NY))
    res = {}
    for split in (1, 0):
        h = handle(n_inner=6, check_every=0, tv_split=split)
        x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
        h.solve(b, 0.01, 0.005, 4, x)
        res[split] = x.cpu()
        if split:
            xb = torch.empty_like(x)
            Batch([h]).solve([b], 0.01, 0.005, 4, [xb])
            assert torch.equal(xb.cpu(), res[1])
        h.close()
    # the split only reorders the restart product's sum
    assert rel_l2(res[1].numpy(), res[0].numpy()) <= 1e-6

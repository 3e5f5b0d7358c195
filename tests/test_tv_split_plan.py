"""The split rule of the two-step TV launches (rihv_tv_split_plan, host only):
with one CTA per SM, a launch whose equal z-chunks leave the last wave partly
idle cuts the z-chunks of its last tiles. Checked here against a separate
list-scheduling model of the launch (a CTA of c planes costs c + halo plane
ticks; CTAs start in launch order on the first free SM) and the rule's
search: the last r tiles (r = 2, 4, ... up to two waves) cut into m = 2, 3
or 4 chunks of at least 8 planes, the shortest modelled makespan kept when
it saves at least 2 %."""
import heapq

import pytest

from paper_1904_04884_gb300.rihv import RihvError, rihv_tv_split_plan

SMS = 152


def tiles(nx, ny, final):
    tx, ty = (58, 11) if final else (60, 16)
    return -(-nx // tx) * -(-ny // ty)


def makespan(ntiles, nz, zc, halo, ka, zc2, sms=SMS):
    free = [0] * sms
    order = [(ka, zc)] + ([(ntiles - ka, zc2)] if zc2 else [])
    for count, c in order:
        for z0 in range(0, nz, c):
            cost = min(c, nz - z0) + halo
            for _ in range(count):
                heapq.heappush(free, heapq.heappop(free) + cost)
    return max(free)


def plan(nx, ny, nz, final, zc, sms=SMS):
    zc = min(zc, nz)
    nt, halo = tiles(nx, ny, final), 4 if final else 3
    base = best = makespan(nt, nz, zc, halo, nt, 0, sms)
    choice = (0, 0)
    step = max(1, sms // 64)
    for m in (2, 3, 4):
        zc2 = -(-zc // m)
        if zc2 < 8:
            break
        for r in range(step, min(nt, 2 * sms) + 1, step):
            t = makespan(nt, nz, zc, halo, nt - r, zc2, sms)
            if t < best:
                best, choice = t, (nt - r, zc2)
    return choice if best * 100 <= base * 98 else (0, 0)


CASES = [(1024, 1024, 256, 256), (512, 512, 700, 235), (512, 512, 128, 128),
         (256, 1024, 32, 32), (768, 768, 192, 96), (256, 256, 64, 13)]


@pytest.mark.parametrize("final", [0, 1])
@pytest.mark.parametrize("nx,ny,nz,zc", CASES)
def test_plan_matches_the_model(nx, ny, nz, zc, final):
    got = rihv_tv_split_plan(nx, ny, nz, final, zc)
    assert got == plan(nx, ny, nz, final, zc)
    split, zc2 = got
    if zc2:
        nt, halo = tiles(nx, ny, final), 4 if final else 3
        assert 0 <= split < nt and 8 <= zc2 < min(zc, nz)
        assert makespan(nt, nz, min(zc, nz), halo, split, zc2) * 100 <= \
            makespan(nt, nz, min(zc, nz), halo, nt, 0) * 98


def test_plans_of_the_workloads():
    # 1024 x 1024 x 256: the last 112 of 1,152 tiles in 86-plane chunks; the
    # fused-final launch's last 20 of 1,692 tiles in 64-plane chunks
    assert rihv_tv_split_plan(1024, 1024, 256, 0, 256) == (1040, 86)
    assert rihv_tv_split_plan(1024, 1024, 256, 1, 256) == (1672, 64)
    # 512 x 512 x 128: 288 CTAs in two nearly full waves, kept equal
    assert rihv_tv_split_plan(512, 512, 128, 0, 128) == (0, 0)


def test_invalid_arguments():
    for args in ((0, 64, 8, 0, 8), (64, 64, 8, 2, 8), (64, 64, 8, 0, 0)):
        with pytest.raises(RihvError):
            rihv_tv_split_plan(*args)
    with pytest.raises(RihvError):
        rihv_tv_split_plan(64, 64, 8, 0, 8, sms=0)

"""Host logic: the level planner (Sec. 3.1, Fig. 3), run on the CPU through
the C ABI.  rhif_plan_selfcheck builds every level with seeded synthetic
survivors and checks the plans against the definitions recomputed from DOF
coordinates (bucket order by code, cells and adjacent separator segments,
group-to-cell lists, extend-add maps landing on the same DOF, identical
rebuild from recycled storage).  No GPU is used."""
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def lib():
    import shutil
    import os
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build the library")
    import paper_1808_01364_gb300 as rhif
    rhif.load()
    return rhif


@pytest.mark.parametrize("ns,leaf,keep,edge", [
    ((63, 63), 8, 0.6, False),        # power-of-two-minus-one grid
    ((100, 37), 8, 0.3, False),       # ragged, unequal sides
    ((255, 255), 16, 0.5, False),
    ((64, 64), 8, 0.0, False),        # every skeletonized DOF dropped
    ((65, 33), 4, 1.0, False),        # nothing dropped
    ((1, 40), 4, 0.5, False),         # degenerate: one column of DOFs
    ((15, 15, 15), 4, 0.5, False),
    ((31, 20, 17), 4, 0.4, True),     # 3D, faces and edges skeletonized
    ((23, 23, 23), 8, 0.7, True),
])
def test_plans_match_their_definitions(lib, ns, leaf, keep, edge):
    levels = lib.rhif_plan_selfcheck(ns, leaf, keep=keep, seed=7, edge_skel_3d=edge)
    assert levels >= 2


def test_large_2d_grid_plans(lib):
    # the 1023^2 benchmark grid: the parallel planner on every level
    assert lib.rhif_plan_selfcheck((1023, 1023), 16, keep=0.55, seed=3) == 7


def test_bad_arguments_are_rejected(lib):
    with pytest.raises(lib.RhifError) as e:
        lib.rhif_plan_selfcheck((10, 10), 1)
    assert e.value.code == -1
    with pytest.raises(lib.RhifError):
        lib.rhif_plan_selfcheck((10, 10), 4, keep=1.5)


def test_concurrent_planners_share_the_host_pool(lib):
    """Batched factorizations plan several problems on concurrent host threads
    that share the planner's thread pool (a caller that finds it busy runs its
    loops itself): every concurrent plan must still match its definitions."""
    from concurrent.futures import ThreadPoolExecutor
    cases = [((255, 255), 8), ((300, 211), 8), ((127, 127), 8), ((400, 97), 16),
             ((63, 63, 63), 8), ((511, 300), 8), ((31, 20, 17), 4), ((200, 200), 16)]
    with ThreadPoolExecutor(max_workers=len(cases)) as ex:
        futs = [ex.submit(lib.rhif_plan_selfcheck, ns, leaf, 0.5, 11 + i, len(ns) == 3)
                for i, (ns, leaf) in enumerate(cases)]
        levels = [f.result() for f in futs]
    assert all(lv >= 2 for lv in levels)

"""The closed loop of Algs. 2-3 on the GPU: every cycle runs one library frame (clear,
insert the arm and the obstacle cloud, EDT of both maps, sphere queries) and one step of
the task-priority controller.  With the avoidance tasks the bounding spheres stay clear
of a sphere obstacle sweeping through the arm; without them the obstacle hits the arm."""
import pytest

from paper_2407_02363_b300 import control
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [3, 7])
def test_closed_loop_avoids_the_sweeping_obstacle(seed):
    v = lib()
    with_tasks = control.run_closed_loop(v, seed=seed, avoid=True)
    without = control.run_closed_loop(v, seed=seed, avoid=False)
    assert with_tasks["min_clearance_m"] > 0.0
    assert without["min_clearance_m"] < -0.05


def test_closed_loop_with_obb_sphere_rows():
    """The same loop with the bounding spheres of Sec. III-B (one row per link OBB)."""
    v = lib()
    with_tasks = control.run_closed_loop(v, seed=3, avoid=True, sphere_rule="obb")
    without = control.run_closed_loop(v, seed=3, avoid=False, sphere_rule="obb")
    assert with_tasks["spheres"] > 7
    assert with_tasks["min_clearance_m"] > 0.0
    assert without["min_clearance_m"] < -0.05

"""Staged upload of the velocity field (pic_stage_velocity_dofs /
pic_commit_velocity_dofs): a field staged on a copy stream while the
particles advance, then committed, gives exactly the run in which the same
field was set directly before each step."""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W
import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1612_03369_gb300 import pic

    return pic


def test_staged_fields_match_direct_sets(P):
    import torch

    wl = W.curl_cube(6, 6, 4, 3)
    fields = [wl.U, 0.7 * wl.U, -0.4 * wl.U, 1.1 * wl.U]
    pinned = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f in fields]
    # direct: set, then step
    mesh_a, a = H.gpu_seed(wl)
    for f in pinned:
        P.pic_set_velocity_dofs(mesh_a.h, f)
        a.advect(wl.dt, 4, 1)
    # staged: the next field is copied on another stream while the step runs
    mesh_b, b = H.gpu_seed(wl)
    cs = torch.cuda.Stream()
    P.pic_stage_velocity_dofs(mesh_b.h, pinned[0], cs)
    P.pic_commit_velocity_dofs(mesh_b.h)
    for n in range(len(pinned)):
        b.advect(wl.dt, 4, 1)
        if n + 1 < len(pinned):
            P.pic_stage_velocity_dofs(mesh_b.h, pinned[n + 1], cs)
            P.pic_commit_velocity_dofs(mesh_b.h)
    torch.cuda.synchronize()
    ga, gb = H.gpu_state(a), H.gpu_state(b)
    for k in ("id", "cell", "x", "xhat", "props"):
        np.testing.assert_array_equal(ga[k], gb[k])


def test_staging_state_errors(P):
    import torch

    wl = W.curl_cube(3, 2, 1, 1)
    X = wl.X
    mesh = P.Mesh(wl.n, X)
    Ud = torch.as_tensor(wl.U, device="cuda")
    with pytest.raises(P.PicError):
        P.pic_stage_velocity_dofs(mesh.h, Ud)  # no first field yet
    mesh.set_velocity(wl.U)
    with pytest.raises(P.PicError):
        P.pic_commit_velocity_dofs(mesh.h)  # nothing staged
    P.pic_stage_velocity_dofs(mesh.h, Ud)
    with pytest.raises(P.PicError):
        P.pic_stage_velocity_dofs(mesh.h, Ud)  # one pending already
    P.pic_commit_velocity_dofs(mesh.h)
    torch.cuda.synchronize()

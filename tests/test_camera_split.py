"""Forward + backward over cameras split across ranks (the one exchange of the multi-GPU path):
two processes share the one GPU, each renders three of six surround cameras of the compositional
scene and back-propagates its own cameras' upstream gradient, then the per-octree gradients are
summed across the two ranks (gloo, through host memory).  The sum must equal the gradient of one
process rendering all six cameras in one call, under the gradient rule of the parity tests.  The
two processes' kernels never wait on one another (each one's only waits are inside its own sorts)."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_CAM, W, H = 6, 480, 270


def _scene():
    import synth
    sc = synth.street_scene(200_000, [20_000] * 3, 3)
    cams = synth.surround_cameras(W, H, n=N_CAM)
    return sc, cams


def _upstream(cam_ids, device):
    import torch
    parts = []
    for c in cam_ids:
        g = torch.Generator().manual_seed(1000 + c)
        parts.append((torch.randn((W * H, 3), generator=g), 0.01 * torch.randn((W * H,), generator=g),
                      torch.randn((W * H,), generator=g)))
    return [torch.cat([p[i] for p in parts]).to(device) for i in range(3)]


def _grads(cam_ids):
    import torch
    import paper_2606_23031_gb300 as dv
    sc, cams = _scene()
    ds = [dv.DeviceOctree.from_host(o) for o in sc.octrees]
    _, _, _, st = dv.dv_render(ds, sc.poses, [cams[c] for c in cam_ids], dv.make_opts(1, 1e-4), save_state=True)
    g_rgb, g_d, g_a = _upstream(cam_ids, "cuda")
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    dv.dv_render_backward(st, g_rgb, g_d, g_a, d_dens, d_sh)
    st.check(wait=True)
    st.free()
    return d_dens, d_sh


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import paper_2606_23031_gb300 as dv
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d_dens, d_sh = _grads(dv.camera_shard(range(N_CAM), rank, world))
    dv.allreduce_gradients(d_dens + d_sh)
    torch.cuda.synchronize()
    q.put((rank, [t.cpu().numpy() for t in d_dens], [t.cpu().numpy() for t in d_sh]))
    dist.barrier()
    dist.destroy_process_group()


def test_camera_split_backward_equals_single_process(dv):
    import torch.multiprocessing as mp
    from helpers import check_grads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=600) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref_d, ref_s = _grads(list(range(N_CAM)))
    ref_d = [t.cpu().numpy() for t in ref_d]
    ref_s = [t.cpu().numpy() for t in ref_s]
    assert sum(np.count_nonzero(x) for x in ref_d) > 1000
    for rank, got_d, got_s in res:
        check_grads(got_d, ref_d, f"rank {rank} d_dens (3 + 3 cameras summed)")
        check_grads(got_s, ref_s, f"rank {rank} d_sh (3 + 3 cameras summed)")

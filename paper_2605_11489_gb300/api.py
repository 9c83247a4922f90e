"""Torch-facing wrapper of the C ABI: device memory and streams come from
PyTorch, every computation runs in libgsr.so.

    ctx = Context()                       # gs_context on the current device
    scene = Scene.from_arrays(synth.tiny_scene())
    out = ctx.forward(scene, cam)         # dict of planar fp32 tensors
    rgb, dcdx, dcdy, depth, alpha = render(ctx, scene.params(), cam)   # autograd

Layouts (include/gsr.h): scene planes [rows, n_pad] fp32 (16-byte aligned,
n_pad % 4 == 0); images planar [3, H, W] / [H, W] fp32.
"""
from __future__ import annotations

import ctypes as C
import glob
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import abi
from .abi import GsCamera, GsOutputs, GsRenderOpts, GsScene, GsSceneGrads, GsStateView, check

OUTPUT_KEYS = ("rgb", "dcdx", "dcdy", "depth", "alpha")
# RaDe-GS channels (plain forward only): the normal channel, the normal-view map and the
# ray-Gaussian intersection depth
NORMAL_KEYS = ("normal", "nv", "depth_isect")


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


@dataclass
class Scene:
    """Gaussians resident on the device, attribute-planar (see include/gsr.h)."""
    n: int
    deg: int
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    logits: torch.Tensor
    sh: torch.Tensor

    @property
    def n_pad(self) -> int:
        return self.means.shape[1]

    @staticmethod
    def from_arrays(s, device="cuda") -> "Scene":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return Scene(s.n, s.deg, t(s.means), t(s.log_scales), t(s.quats), t(s.logits), t(s.sh))

    @staticmethod
    def from_tensors(n, deg, means, log_scales, quats, logits, sh) -> "Scene":
        return Scene(n, deg, means, log_scales, quats, logits, sh)

    def params(self):
        return self.means, self.log_scales, self.quats, self.logits, self.sh

    def struct(self) -> GsScene:
        for t in self.params():
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("scene planes must be contiguous fp32 CUDA tensors")
        return GsScene(self.n, self.n_pad, self.deg, 0, _ptr(self.means), _ptr(self.log_scales), _ptr(self.quats),
                       _ptr(self.logits), _ptr(self.sh))

    def zeros_like_grads(self):
        return tuple(torch.zeros_like(t) for t in self.params())


def camera_struct(cam) -> GsCamera:
    c = GsCamera()
    for k in range(12):
        c.viewmat[k] = float(cam.viewmat[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def opts_struct(tile=0, batch=0, bg=(0.0, 0.0, 0.0), state=False, timed=False, chunk=0, count=False,
                head=0) -> GsRenderOpts:
    o = GsRenderOpts()
    o.tile, o.batch, o.chunk, o.head = int(tile), int(batch), int(chunk), int(head)
    for k in range(3):
        o.bg[k] = float(bg[k])
    # timed: True = events at every stage boundary, "composite" = around compositing only
    tflag = abi.GS_TIME_COMPOSITE if timed == "composite" else (abi.GS_TIME_STAGES if timed else 0)
    o.flags = (abi.GS_EMIT_BWD_STATE if state else 0) | tflag | (abi.GS_COUNT_PAIRS if count else 0)
    return o


def _stats_dict(st) -> dict:
    return dict(frames=st.frames, instances_total=st.instances_total, visible_total=st.visible_total,
                instances_max=st.instances_max, timed_frames=st.timed_frames,
                pairs_evaluated=st.pairs_evaluated, pairs_blended=st.pairs_blended,
                stage_ms={k: st.stage_ms[i] for i, k in enumerate(abi.STAGES)})


def alloc_outputs(width, height, keys=OUTPUT_KEYS, device="cuda") -> dict:
    shp = {"rgb": (3, height, width), "dcdx": (3, height, width), "dcdy": (3, height, width),
           "depth": (height, width), "alpha": (height, width), "normal": (3, height, width), "nv": (height, width),
           "depth_isect": (height, width)}
    return {k: torch.empty(shp[k], dtype=torch.float32, device=device) for k in keys}


WARP_KEYS = ("motion", "index", "z", "planes", "dcdx", "dcdy")


def alloc_warp_outputs(width, height, width_t, height_t, channels, grad_channels, keys=WARP_KEYS,
                       device="cuda") -> dict:
    """Target planes of gs_warp (and the source-sized motion map)."""
    shp = {"motion": ((2, height, width), torch.float32), "index": ((height_t, width_t), torch.int32),
           "z": ((height_t, width_t), torch.float32), "planes": ((channels, height_t, width_t), torch.float32),
           "dcdx": ((grad_channels, height_t, width_t), torch.float32),
           "dcdy": ((grad_channels, height_t, width_t), torch.float32)}
    return {k: torch.empty(shp[k][0], dtype=shp[k][1], device=device) for k in keys}


def outputs_struct(out: dict) -> GsOutputs:
    return GsOutputs(*[_ptr(out.get(k)) for k in OUTPUT_KEYS + NORMAL_KEYS])


# ----------------------------------------------------------------------------- raw device copies (inspection)
_cudart = None


def _cudart_lib():
    global _cudart
    if _cudart is None:
        cands = []
        tdir = os.path.dirname(torch.__file__)
        cands += glob.glob(os.path.join(os.path.dirname(tdir), "nvidia", "cu*", "lib", "libcudart.so*"))
        cands += glob.glob(os.path.join(os.path.dirname(tdir), "nvidia", "cuda_runtime", "lib", "libcudart.so*"))
        cands += glob.glob(os.path.join(tdir, "lib", "libcudart*.so*"))
        cands += glob.glob("/usr/local/cuda/lib64/libcudart.so*")
        for c in cands:
            try:
                _cudart = C.CDLL(c)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("libcudart not found")
        _cudart.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        _cudart.cudaMemcpy.restype = C.c_int
    return _cudart


def device_to_numpy(ptr: int, count: int, dtype) -> np.ndarray:
    """Copy `count` elements of `dtype` from a raw device pointer (synchronous)."""
    torch.cuda.synchronize()
    a = np.empty(max(int(count), 0), dtype=dtype)
    if count > 0:
        rc = _cudart_lib().cudaMemcpy(a.ctypes.data, ptr, a.nbytes, 2)
        if rc != 0:
            raise RuntimeError("cudaMemcpy failed: %d" % rc)
    return a


# ----------------------------------------------------------------------------- context
class State:
    """Buffers a forward kept for the backward pass (gs_fwd_state)."""

    def __init__(self, handle: int, cam):
        self.handle = C.c_void_p(handle)
        self.cam = cam

    def view(self) -> dict:
        v = GsStateView()
        check(abi.lib().gs_state_view_get(self.handle, C.byref(v)))
        K = v.n_instances
        hw = self.cam.width * self.cam.height
        out = dict(n_instances=K, n_tiles=v.n_tiles, tiles_x=v.tiles_x, tiles_y=v.tiles_y, tile=v.tile,
                   keys=device_to_numpy(v.keys, K, np.uint64), vals=device_to_numpy(v.vals, K, np.uint32),
                   ranges=device_to_numpy(v.ranges, 2 * v.n_tiles, np.uint32).reshape(-1, 2))
        if v.final_T:
            out["final_T"] = device_to_numpy(v.final_T, hw, np.float32).reshape(self.cam.height, self.cam.width)
            out["n_contrib"] = device_to_numpy(v.n_contrib, hw, np.uint32).reshape(self.cam.height, self.cam.width)
        out["_records_ptr"] = v.records
        out["_ntiles_ptr"] = v.ntiles
        return out

    def records(self, n: int) -> np.ndarray:
        v = GsStateView()
        check(abi.lib().gs_state_view_get(self.handle, C.byref(v)))
        return device_to_numpy(v.records, 12 * n, np.float32).reshape(n, 12)

    def ntiles(self, n: int) -> np.ndarray:
        v = GsStateView()
        check(abi.lib().gs_state_view_get(self.handle, C.byref(v)))
        return device_to_numpy(v.ntiles, n, np.uint32)

    def free(self):
        if self.handle:
            abi.lib().gs_state_free(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A gs_context: owns the render workspace on one device."""

    def __init__(self, device: int | None = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        check(abi.lib().gs_context_create(self.device, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            abi.lib().gs_context_destroy(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, scene: Scene, cam, tile=0, batch=0, bg=(0.0, 0.0, 0.0), keys=OUTPUT_KEYS, out=None,
                state=False, timed=False, stream=None, chunk=0, count=False, head=0):
        """Render; returns the output dict (and a State if state=True)."""
        if out is None:
            out = alloc_outputs(cam.width, cam.height, keys)
        sc, cm = scene.struct(), camera_struct(cam)
        op, ou = opts_struct(tile, batch, bg, state, timed, chunk, count, head), outputs_struct(out)
        hs = C.c_void_p()
        check(abi.lib().gs_render_forward(self.h, C.byref(sc), C.byref(cm), C.byref(op), C.byref(ou),
                                          C.byref(hs) if state else None, _stream_ptr(stream)))
        if state:
            return out, State(hs.value, cam)
        return out

    def forward_to_host(self, scene: Scene, cam, host_out: dict, tile=0, batch=0, bg=(0.0, 0.0, 0.0), stream=None):
        """Render into HOST tensors (pinned recommended); synchronous."""
        for t in host_out.values():
            if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32:
                raise ValueError("host outputs must be contiguous fp32 CPU tensors")
        sc, cm, op, ou = scene.struct(), camera_struct(cam), opts_struct(tile, batch, bg), outputs_struct(host_out)
        check(abi.lib().gs_render_forward_to_host(self.h, C.byref(sc), C.byref(cm), C.byref(op), C.byref(ou),
                                                  _stream_ptr(stream)))
        return host_out

    def backward(self, state: State, scene: Scene, grads_in: dict, grads=None, stream=None):
        """Adds d(sum <grads_in, outputs>)/d(params) into `grads` (zeros if None)."""
        if grads is None:
            grads = scene.zeros_like_grads()
        gi = outputs_struct(grads_in)
        go = GsSceneGrads(*[_ptr(g) for g in grads])
        sc = scene.struct()
        check(abi.lib().gs_render_backward(self.h, state.handle, C.byref(sc), C.byref(gi), C.byref(go),
                                           _stream_ptr(stream)))
        return grads

    def warp(self, src_cam, dst_cam, depth, alpha=None, alpha_min=0.0, planes=None, dcdx=None, dcdy=None,
             out=None, keys=WARP_KEYS, stream=None) -> dict:
        """Frame-interpolation warp of one source frame toward ``dst_cam`` (gs_warp):
        motion vectors, the depth-tested forward warp of ``planes`` and the warped
        gradient of (dcdx, dcdy). Inputs are device tensors [H, W] / [C, H, W]; returns
        (or fills) the dict of target planes named in ``keys``."""
        H, W, Ht, Wt = src_cam.height, src_cam.width, dst_cam.height, dst_cam.width
        C_ = 0 if planes is None else int(planes.shape[0])
        G = 0 if dcdx is None else int(dcdx.shape[0])
        for t in (depth, alpha, planes, dcdx, dcdy):
            if t is not None and not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("warp inputs must be contiguous fp32 CUDA tensors")
        if out is None:
            out = alloc_warp_outputs(W, H, Wt, Ht, C_, G, keys)
        gi = abi.GsWarpInput(_ptr(depth), _ptr(alpha), float(alpha_min), C_, _ptr(planes), G, _ptr(dcdx), _ptr(dcdy))
        go = abi.GsWarpOutput(*[_ptr(out.get(k)) for k in WARP_KEYS])
        sc, dc = camera_struct(src_cam), camera_struct(dst_cam)
        check(abi.lib().gs_warp(self.h, C.byref(sc), C.byref(dc), C.byref(gi), C.byref(go), _stream_ptr(stream)))
        return out

    def stats(self, reset=False, stream=None) -> dict:
        st = abi.GsFrameStats()
        check(abi.lib().gs_context_stats(self.h, _stream_ptr(stream), int(reset), C.byref(st)))
        return _stats_dict(st)

    def check(self, stream=None) -> int:
        """Device error status of the plain frames since the last report (gs_context_check):
        returns the status code (0 = GS_OK) without raising."""
        return abi.lib().gs_context_check(self.h, _stream_ptr(stream))

    def debug_waits(self, give_up) -> None:
        """Diagnostic (gs_context_debug_waits): make the bounded device waits of the later
        plain forwards give up at once, to exercise the GS_ERR_TIMEOUT path: 1 (or True)
        every wait, 2 compositing's batch waits only, 0 (or False) none."""
        check(abi.lib().gs_context_debug_waits(self.h, int(give_up)))

    def graph(self, scene: Scene, cam, out: dict, capacity=0, tile=0, batch=0, bg=(0.0, 0.0, 0.0), timed=False,
              stream=None, chunk=0, head=0):
        return Graph(self, scene, cam, out, capacity, tile, batch, bg, stream, timed, chunk, head)

    def autotune(self, scene: Scene, cam, out: dict, iters=3, stream=None):
        """Returns (tile, batch, chunk, ms) of the fastest configuration, now cached."""
        t, b, k, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float()
        sc, cm, ou = scene.struct(), camera_struct(cam), outputs_struct(out)
        check(abi.lib().gs_autotune(self.h, C.byref(sc), C.byref(cm), C.byref(ou), int(iters), _stream_ptr(stream),
                                    C.byref(t), C.byref(b), C.byref(k), C.byref(ms)))
        return t.value, b.value, k.value, ms.value


class Graph:
    """Captured whole-frame forward replayed with a new camera per frame."""

    def __init__(self, ctx: Context, scene: Scene, cam, out: dict, capacity, tile, batch, bg, stream, timed=False,
                 chunk=0, head=0):
        self.ctx, self.scene, self.out = ctx, scene, out  # keep the buffers alive
        sc, cm = scene.struct(), camera_struct(cam)
        op, ou = opts_struct(tile, batch, bg, timed=timed, chunk=chunk, head=head), outputs_struct(out)
        h = C.c_void_p()
        check(abi.lib().gs_graph_create(ctx.h, C.byref(sc), C.byref(cm), C.byref(op), C.byref(ou), int(capacity),
                                        _stream_ptr(stream), C.byref(h)))
        self.h = h

    def render(self, cam, stream=None):
        cm = camera_struct(cam)
        check(abi.lib().gs_graph_render(self.h, C.byref(cm), _stream_ptr(stream)))

    def check(self, stream=None) -> int:
        mx = C.c_int64()
        check(abi.lib().gs_graph_check(self.h, _stream_ptr(stream), C.byref(mx)))
        return mx.value

    def stats(self, reset=False, stream=None) -> dict:
        st = abi.GsFrameStats()
        check(abi.lib().gs_graph_stats(self.h, _stream_ptr(stream), int(reset), C.byref(st)))
        return _stats_dict(st)

    def close(self):
        if self.h:
            abi.lib().gs_graph_destroy(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching render server (gs_server_*)."""

    def __init__(self, device: int | None = None, sort_budget_bytes: int = 1 << 30, max_inflight: int = 8):
        dev = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        check(abi.lib().gs_server_create(dev, C.c_size_t(int(sort_budget_bytes)), int(max_inflight), C.byref(h)))
        self.h = h
        self._keep = {}

    def load_scene(self, scene: Scene) -> int:
        sid = C.c_int32()
        sc = scene.struct()
        torch.cuda.synchronize()
        check(abi.lib().gs_server_load_scene(self.h, C.byref(sc), C.byref(sid)))
        return sid.value

    def submit(self, scene_id: int, cam, out: dict, bg=(0.0, 0.0, 0.0)) -> int:
        rid = C.c_uint64()
        cm, op, ou = camera_struct(cam), opts_struct(0, 0, bg), outputs_struct(out)
        check(abi.lib().gs_server_submit(self.h, int(scene_id), C.byref(cm), C.byref(op), C.byref(ou), C.byref(rid)))
        self._keep[rid.value] = out
        return rid.value

    def poll(self, rid: int):
        """Returns (status, latency_ms); status GS_NOT_READY while in flight."""
        lat = C.c_double()
        st = abi.lib().gs_server_poll(self.h, C.c_uint64(rid), C.byref(lat))
        if st != abi.GS_NOT_READY:
            self._keep.pop(rid, None)
        return st, lat.value

    def cancel(self, rid: int) -> int:
        return abi.lib().gs_server_cancel(self.h, C.c_uint64(rid))

    def drain(self):
        check(abi.lib().gs_server_drain(self.h))

    def close(self):
        if self.h:
            abi.lib().gs_server_destroy(self.h)
            self.h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- gradient-aware interpolation
def gai_upsample(weights, rgb, dcdx, dcdy, out=None, stream=None):
    """Super-sampling by the gradient-aware interpolation of Sec. 4.1 (gs_gai_upsample).

    weights: (scale, wc [C, 27], bc [C] or None, wt [S*S, C], bt [S*S] or None), host
    arrays of the Conv3x3 -> SxS TConv of Eq. 8. rgb, dcdx, dcdy: device [channels, H, W]
    fp32. Returns (or fills) out [channels, S H, S W]."""
    S, wc, bc, wt, bt = weights
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    wc, bc, wt, bt = f32(wc), f32(bc), f32(wt), f32(bt)
    Cf = wc.shape[0]
    if wc.shape != (Cf, 27) or wt.shape != (S * S, Cf):
        raise ValueError("weights must be wc [C, 27] and wt [S*S, C]")
    for t in (rgb, dcdx, dcdy):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.shape == rgb.shape):
            raise ValueError("rgb, dcdx, dcdy must be contiguous fp32 CUDA tensors of one shape")
    ch, H, W = rgb.shape
    if out is None:
        out = torch.empty((ch, S * H, S * W), dtype=torch.float32, device=rgb.device)
    hp = lambda a: None if a is None else a.ctypes.data
    w = abi.GsGaiWeights(int(S), int(Cf), hp(wc), hp(bc), hp(wt), hp(bt))
    check(abi.lib().gs_gai_upsample(C.byref(w), _ptr(rgb), _ptr(dcdx), _ptr(dcdy), int(ch), int(W), int(H),
                                    _ptr(out), _stream_ptr(stream)))
    return out


# ----------------------------------------------------------------------------- frames to the host
class FrameStream:
    """Renders a camera sequence on the device with `slots` frames in flight (default 2),
    through the C ABI's frame stream (gs_frame_stream_*).
    - One captured graph per slot, each with its own output buffers (`outs[k]`) and its own
      high-priority stream, takes the frames in turn. Consecutive frames are independent,
      so one frame's compositing runs beside the next frames' projection and sorts.
    - `render(cam)` returns the slot k that frame goes to. `wait_for(k, stream)` makes a
      stream wait until slot k's latest frame has rendered; then `outs[k]` may be read there.
    - A consumer that reads `outs[k]` on its own stream calls `release(k, stream)` when it
      has enqueued those reads. The next frame rendered into slot k then waits for them.
      Without a release, slot k is rewritten `slots` frames later.
    Every computation, stream and event lives in libgsr.so."""

    def __init__(self, ctx: "Context", scene: "Scene", cam0, capacity: int, tile=0, batch=0, chunk=0,
                 keys=OUTPUT_KEYS, timed=False, slots=2):
        W, H = cam0.width, cam0.height
        self.slots = n = int(slots)
        if n < 1:
            raise ValueError("slots must be >= 1")
        self.ctx, self.scene = ctx, scene  # keep alive
        self.outs = [alloc_outputs(W, H, tuple(keys)) for _ in range(n)]
        sets = (GsOutputs * n)(*[outputs_struct(o) for o in self.outs])
        op = opts_struct(tile, batch, (0.0, 0.0, 0.0), timed=timed, chunk=chunk)
        h = C.c_void_p()
        torch.cuda.synchronize()
        check(abi.lib().gs_frame_stream_create(ctx.h, C.byref(scene.struct()), C.byref(camera_struct(cam0)),
                                               C.byref(op), sets, n, int(capacity), C.byref(h)))
        self.h = h
        self.frame = [-1] * n  # the latest frame number of each slot

    def render(self, cam, host_out: dict = None) -> int:
        """Enqueue frame `cam`; with `host_out` (pinned fp32 CPU tensors keyed like `outs`)
        its planes are also copied there after the render."""
        f = C.c_int64()
        ho = C.byref(outputs_struct(host_out)) if host_out is not None else None
        check(abi.lib().gs_frame_stream_submit(self.h, C.byref(camera_struct(cam)), ho, C.byref(f)))
        k = f.value % self.slots
        self.frame[k] = f.value
        return k

    def wait_for(self, k: int, stream) -> None:
        check(abi.lib().gs_frame_stream_join(self.h, self.frame[k], _stream_ptr(stream)))

    def release(self, k: int, stream) -> None:
        check(abi.lib().gs_frame_stream_release(self.h, self.frame[k], _stream_ptr(stream)))

    def follow(self, stream) -> None:
        """Every slot's next frame waits for the work enqueued on `stream` so far."""
        for k in range(self.slots):
            if self.frame[k] >= 0:
                self.release(k, stream)

    def join(self, stream) -> None:
        """Makes `stream` wait for every frame submitted so far."""
        for k in range(self.slots):
            if self.frame[k] >= 0:
                self.wait_for(k, stream)

    def synchronize(self) -> None:
        """Waits for every submitted frame; raises if a frame overflowed the graphs'
        instance capacity or a bounded wait gave up."""
        check(abi.lib().gs_frame_stream_synchronize(self.h))

    def stats(self, reset=False) -> list:
        out = []
        for k in range(self.slots):
            st = abi.GsFrameStats()
            check(abi.lib().gs_frame_stream_stats(self.h, k, int(reset), C.byref(st)))
            out.append(_stats_dict(st))
        return out

    def close(self) -> None:
        if self.h:
            self.synchronize()
            abi.lib().gs_frame_stream_destroy(self.h)
            self.h = C.c_void_p(0)


class HostFrameStream(FrameStream):
    """Renders a camera sequence into HOST planes (pinned memory) through the C ABI's frame
    stream: each frame's device-to-host copies run on its slot's stream right after its
    render, beside the other slots' renders. The caller owns the host buffers and must not
    touch a frame's buffers until `synchronize()`."""

    def __init__(self, ctx: "Context", scene: "Scene", cam0, capacity: int, tile=0, batch=0, chunk=0,
                 keys=OUTPUT_KEYS, slots=2):
        super().__init__(ctx, scene, cam0, capacity, tile, batch, chunk, keys, False, slots)

    def render(self, cam, host_out: dict) -> int:
        """Enqueue frame `cam`; its planes land in `host_out` (pinned fp32 CPU tensors of
        the output shapes, keyed like the device outputs)."""
        return super().render(cam, host_out)


# ----------------------------------------------------------------------------- pipeline
class FramePipeline:
    """The post-rendering chain of Sec. 4, with the low-resolution render of the next frame
    overlapping the super-sampling and interpolation inputs of the current one (Sec. 5.1:
    super sampling and frame interpolation run in parallel; the pipeline-parallel deployment
    of Sec. 5.4).

    Per frame t (camera cams[t]; mid = the pose between frames t - 1 and t):
      render streams: frame t's colour, gradients, depth and alpha at low resolution
                      (a captured graph per output buffer; `slots` buffers in turn, each on
                      its own stream, so consecutive renders overlap too)
      post stream:    x S gradient-aware interpolation of the colour (Sec. 4.1) and of depth
                      and alpha (no gradients: a linear filter of the values);
                      forward warp of the x S frame t - 1 toward the mid pose (Sec. 4.2);
                      backward warp of the low-resolution frame t, with its gradients,
                      toward the mid pose.
    Events order the streams: the post chain of frame t waits for its render, and the
    render of frame t + slots waits until the chain of frame t has read their shared buffer.
    overlap=False runs both on one stream (the serial baseline). Every computation runs in
    libgsr.so; this class only orders the calls."""

    # an interpolated pixel moves in the forward warp only where its interpolated alpha
    # exceeds this (the interpolation can leave tiny nonzero values next to empty pixels)
    HR_ALPHA_MIN = 0.01

    def __init__(self, ctx: "Context", scene: "Scene", cam0, gai_weights, capacity: int, tile=0, batch=0,
                 chunk=0, overlap=True, slots=2):
        S = int(gai_weights[0])
        self.slots = n = int(slots) if overlap else 2
        if n < 2:
            raise ValueError("slots must be >= 2")
        W, H = cam0.width, cam0.height
        self.ctx, self.scene, self.weights, self.S = ctx, scene, gai_weights, S
        # the render streams have the higher priority: the post chain's large grids fill the
        # SMs the renders leave idle instead of delaying them
        if overlap:
            self.rs = [torch.cuda.Stream(priority=-1) for _ in range(n)]
            self.ps = torch.cuda.Stream(priority=0)
        else:
            one = torch.cuda.Stream()
            self.rs, self.ps = [one] * n, one
        self.lr, self.da = [], []
        for _ in range(n):
            da = torch.empty((2, H, W), dtype=torch.float32, device="cuda")  # depth, alpha
            out = alloc_outputs(W, H, keys=("rgb", "dcdx", "dcdy"))
            out["depth"], out["alpha"] = da[0], da[1]
            self.lr.append(out)
            self.da.append(da)
        self.zero_g = torch.zeros((2, H, W), dtype=torch.float32, device="cuda")
        self.graphs = [ctx.graph(scene, cam0, self.lr[k], capacity=capacity, tile=tile, batch=batch, chunk=chunk,
                                 stream=self.rs[k]) for k in range(n)]
        self.hr_rgb = [torch.empty((3, S * H, S * W), dtype=torch.float32, device="cuda") for _ in range(n)]
        self.hr_da = [torch.empty((2, S * H, S * W), dtype=torch.float32, device="cuda") for _ in range(n)]
        self.wctx = Context(ctx.device)  # the warps' scratch, used on the post stream only
        self.fwd = alloc_warp_outputs(S * W, S * H, S * W, S * H, 3, 0, keys=("motion", "index", "z", "planes"))
        self.bwd = alloc_warp_outputs(W, H, W, H, 3, 3)
        self.rendered = [torch.cuda.Event() for _ in range(n)]
        self.consumed = [torch.cuda.Event() for _ in range(n)]
        self.used = [False] * n
        self.prev_cam = None
        torch.cuda.synchronize()

    def step(self, cam, mid):
        """Frame `cam` through the chain; `mid` is the pose between the previous frame and it.
        Asynchronous: after it, the post stream holds this frame's interpolated colour
        (hr_rgb[k]), depth and alpha (hr_da[k]) and the two warps' outputs (fwd, bwd)."""
        k = 0 if self.prev_cam is None else (self._k + 1) % self.slots
        if self.used[k]:
            self.rs[k].wait_event(self.consumed[k])
        self.graphs[k].render(cam, stream=self.rs[k])
        self.rendered[k].record(self.rs[k])
        self.ps.wait_event(self.rendered[k])
        lr, S = self.lr[k], self.S
        gai_upsample(self.weights, lr["rgb"], lr["dcdx"], lr["dcdy"], out=self.hr_rgb[k], stream=self.ps)
        gai_upsample(self.weights, self.da[k], self.zero_g, self.zero_g, out=self.hr_da[k], stream=self.ps)
        if self.prev_cam is not None:
            j = self._k
            self.wctx.warp(self.prev_cam.scaled(S), mid.scaled(S), self.hr_da[j][0], self.hr_da[j][1],
                           self.HR_ALPHA_MIN, self.hr_rgb[j], out=self.fwd, stream=self.ps)
        self.wctx.warp(cam, mid, lr["depth"], lr["alpha"], 0.0, lr["rgb"], lr["dcdx"], lr["dcdy"], out=self.bwd,
                       stream=self.ps)
        self.consumed[k].record(self.ps)
        self.used[k] = True
        self._k, self.prev_cam = k, cam
        return k

    def synchronize(self):
        for st in self.rs:
            st.synchronize()
        self.ps.synchronize()

    def close(self):
        self.synchronize()
        for g in self.graphs:
            g.close()
        self.wctx.close()


# ----------------------------------------------------------------------------- autograd
class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, means, log_scales, quats, logits, sh, gctx, n, deg, cam, bg, tile, batch):
        scene = Scene(n, deg, means.contiguous(), log_scales.contiguous(), quats.contiguous(), logits.contiguous(),
                      sh.contiguous())
        out, state = gctx.forward(scene, cam, tile=tile, batch=batch, bg=bg, state=True)
        fctx.gctx, fctx.state, fctx.scene = gctx, state, scene
        fctx.mark_non_differentiable()
        return tuple(out[k] for k in OUTPUT_KEYS)

    @staticmethod
    def backward(fctx, g_rgb, g_dcdx, g_dcdy, g_depth, g_alpha):
        gi = {}
        for k, g in zip(OUTPUT_KEYS, (g_rgb, g_dcdx, g_dcdy, g_depth, g_alpha)):
            if g is not None:
                gi[k] = g.contiguous()
        grads = fctx.gctx.backward(fctx.state, fctx.scene, gi)
        fctx.state.free()
        return (*grads, None, None, None, None, None, None, None)


def render(gctx: Context, params, cam, n: int | None = None, deg: int | None = None, bg=(0.0, 0.0, 0.0), tile=0,
           batch=0):
    """Differentiable render: params = (means [3,n_pad], log_scales [3,n_pad], quats [4,n_pad],
    logits [n_pad], sh [K,3,n_pad]); returns (rgb, dcdx, dcdy, depth, alpha)."""
    means, log_scales, quats, logits, sh = params
    if n is None:
        n = means.shape[1]
    if deg is None:
        deg = int(round(sh.shape[0] ** 0.5)) - 1
    return _RenderFn.apply(means, log_scales, quats, logits, sh, gctx, int(n), int(deg), cam, tuple(bg), int(tile),
                           int(batch))

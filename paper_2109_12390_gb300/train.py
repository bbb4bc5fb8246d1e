"""Python surface of decoder training and snapshot generation (argument marshalling only).

Snapshots come from the GPU MPM (csrc/mpm.cu) and stay on the device;
training runs in csrc/train.cu.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from .mpm import MPM, _stream


def _vp(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def generate_snapshots(scene, n_steps, every, device="cuda"):
    """Runs the batched GPU MPM on `scene` (synth.scenes.Scene) and keeps x, v, F at steps
    0, every, 2 every, ... <= n_steps.  Returns a dict of device tensors in the layout of
    snapshot_desc (snapshot s = time j * n_inst + instance k)."""
    ctx = MPM.from_scene(scene)
    ctx.load_numpy(scene.x, scene.v, scene.F, scene.C)
    P, d = scene.n_particles, scene.dim
    J = n_steps // every + 1
    xs = torch.empty((J, P, d), dtype=torch.float32, device=device)
    vs = torch.empty((J, P, d), dtype=torch.float32, device=device)
    Fs = torch.empty((J, P, d * d), dtype=torch.float32, device=device)
    for j in range(J):
        if j > 0:
            ctx.step(every)
        ctx.get_state(xs[j], vs[j], Fs[j], None)
    torch.cuda.synchronize()
    status = ctx.status()
    ctx.close()
    n_inst = scene.n_inst
    S = J * n_inst
    snap_inst = np.array([s % n_inst for s in range(S)], np.int32)
    snap_next = np.array([s + n_inst if s + n_inst < S else -1 for s in range(S)], np.int32)
    return dict(dim=d, n_inst=n_inst, inst_offsets=np.ascontiguousarray(scene.inst_offsets, np.int64),
                X=torch.from_numpy(scene.x.astype(np.float32)).to(device), n_snap=S, snap_inst=snap_inst,
                snap_next=snap_next, x=xs.reshape(-1, d), v=vs.reshape(-1, d), F=Fs.reshape(-1, d * d),
                status=status, steps_between=every, dt_snap=every * float(np.float32(scene.dt)))


def snapshot_desc(snaps):
    """The C snapshot_desc of a snapshot dict (pointers into its arrays, which the caller keeps alive)."""
    return _abi.SnapshotDesc(snaps["dim"], snaps["n_inst"], _vp(snaps["inst_offsets"]), _vp(snaps["X"]),
                             snaps["n_snap"], _vp(snaps["snap_inst"]), _vp(snaps["snap_next"]),
                             _vp(snaps["x"]), _vp(snaps["v"]), _vp(snaps["F"]))


class Trainer:
    def __init__(self, decoder, snaps, *, lambda_F=100.0, lambda_v=0.01, dt_snap, lr0=1e-3, lr1=1e-6,
                 batch=65536, total_steps=10000, seed=0, latents0=None, encoder_subset=0, shard_index=0,
                 shard_count=1):
        """batch: this context's points per step; with shard_count > 1 it is one data-parallel shard
        (draws shard_index * batch ... of a minibatch of shard_count * batch points)."""
        L = _abi.lib()
        self.decoder = decoder
        self.snaps = snaps
        self._keep = [snaps["inst_offsets"], snaps["snap_inst"], snaps["snap_next"]]
        sd = snapshot_desc(snaps)
        cfg = _abi.TrainConfig(lambda_F, lambda_v, dt_snap, lr0, lr1, batch, total_steps, seed, encoder_subset,
                               int(shard_index), int(shard_count))
        self.cfg = cfg
        lat = None if latents0 is None else np.ascontiguousarray(latents0, np.float32)
        h = C.c_void_p()
        _abi.check(L.trainer_create(decoder._h, C.byref(cfg), C.byref(sd), _vp(lat), C.byref(h)))
        self._h = h
        self.n_snap, self.r, self.batch = snaps["n_snap"], decoder.r, batch
        self.encoder_subset = int(encoder_subset)
        self.d = snaps["dim"]

    def close(self):
        if getattr(self, "_h", None):
            _abi.lib().trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_steps=1, stream=None):
        _abi.check(_abi.lib().decoder_train(self._h, int(n_steps), _stream(stream)))

    def gradient_buffers(self):
        """Device tensors sized for this trainer's gradients: (decoder parameters, latent table or
        encoder parameters)."""
        n0, n1 = C.c_int64(), C.c_int64()
        _abi.check(_abi.lib().trainer_gradient_sizes(self._h, C.byref(n0), C.byref(n1)))
        return (torch.empty(n0.value, dtype=torch.float32, device="cuda"),
                torch.empty(n1.value, dtype=torch.float32, device="cuda"))

    def compute_gradients(self, g_params, g_second, stream=None):
        """This shard's forward and backward of the next step: gradients into the two tensors."""
        assert g_params.is_cuda and g_second.is_cuda and g_params.dtype == torch.float32
        _abi.check(_abi.lib().trainer_compute_gradients(self._h, _vp(g_params), _vp(g_second), _stream(stream)))

    def apply_gradients(self, g_params, g_second, stream=None):
        """The Adam step with the given (summed over the shards) gradients."""
        assert g_params.is_cuda and g_second.is_cuda and g_params.dtype == torch.float32
        _abi.check(_abi.lib().trainer_apply_gradients(self._h, _vp(g_params), _vp(g_second), _stream(stream)))

    def loss(self, stream=None):
        l = C.c_double()
        st = C.c_int64()
        _abi.check(_abi.lib().trainer_loss(self._h, C.byref(l), C.byref(st), _stream(stream)))
        return l.value, st.value

    def latents(self, stream=None):
        out = np.empty((self.n_snap, self.r), np.float32)
        _abi.check(_abi.lib().trainer_get_latents(self._h, _vp(out), _stream(stream)))
        torch.cuda.synchronize()
        return out

    def status(self, clear=True, stream=None):
        w = C.c_uint32()
        _abi.check(_abi.lib().trainer_status_word(self._h, C.byref(w), int(clear), _stream(stream)))
        return w.value

    def gradients(self, stream=None):
        """(decoder parameter gradients, per-snapshot latent gradients, batch snapshot ids, batch
        particle ids, loss) of one forward/backward without update; with an encoder, the encoder's
        parameter gradients are in self.last_encoder_gradients."""
        gp = np.empty(self.decoder.n_params, np.float32)
        gl = np.empty((self.n_snap, self.r), np.float32)
        ge = np.empty(self.encoder_n_params(), np.float32) if self.encoder_subset else None
        bs = np.empty(self.batch, np.int32)
        bp = np.empty(self.batch, np.int32)
        loss = C.c_double()
        _abi.check(_abi.lib().trainer_gradients(self._h, _vp(gp), _vp(gl), _vp(ge), _vp(bs), _vp(bp),
                                                C.byref(loss), _stream(stream)))
        self.last_encoder_gradients = ge
        return gp, gl, bs, bp, loss.value

    # ---- encoder (train_config.encoder_subset > 0)
    def encoder_n_params(self):
        n = C.c_int64()
        _abi.check(_abi.lib().trainer_encoder_params(self._h, None, None, C.byref(n), None))
        return n.value

    def encoder_params(self, stream=None):
        """(parameter vector, shift_scale (2 d))"""
        p = np.empty(self.encoder_n_params(), np.float32)
        ss = np.empty(2 * self.d, np.float32)
        _abi.check(_abi.lib().trainer_encoder_params(self._h, _vp(p), _vp(ss), None, _stream(stream)))
        return p, ss

    def set_encoder_params(self, params=None, shift_scale=None, stream=None):
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        ss = None if shift_scale is None else np.ascontiguousarray(shift_scale, np.float32)
        _abi.check(_abi.lib().trainer_set_encoder_params(self._h, _vp(p), _vp(ss), _stream(stream)))

    def encode(self, x, stream=None):
        """x (n, P, d) full-order positions -> (n, r) generalized coordinates."""
        if isinstance(x, torch.Tensor):
            x = x.detach().float().contiguous()
            n, P = x.shape[0], x.shape[1]
        else:
            x = np.ascontiguousarray(x, np.float32)
            n, P = x.shape[0], x.shape[1]
        out = np.empty((n, self.r), np.float32)
        _abi.check(_abi.lib().trainer_encode(self._h, _vp(x), int(n), int(P), _vp(out), _stream(stream)))
        return out

"""ctypes declarations of include/ntbc.h and thin wrappers (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libntbc.so")

BC1, BC4 = 1, 4
BC3, BC5 = 3, 5
ACT_SELU, ACT_RELU = 0, 1
PREC_FP32, PREC_FP16, PREC_FP16_FAST, PREC_FP8, PREC_FP8_MMA = 0, 1, 2, 3, 4
BATCH_CHAINED, BATCH_QUEUE = 0, 1
TRAIN_FP32, TRAIN_BF16 = 0, 1
MAX_TEXTURES, MAX_LEVELS, MAX_MLP_LAYERS = 8, 16, 4
STATUS_NAMES = {0: "NTBC_OK", 1: "NTBC_EINVAL", 2: "NTBC_ENOMEM", 3: "NTBC_ECUDA", 4: "NTBC_ETIMEOUT",
                5: "NTBC_ENONFINITE", 6: "NTBC_EUNSUPPORTED"}

if not os.path.exists(library_path):
    raise ImportError(f"libntbc.so is not built ({library_path}); run __graft_entry__.build() "
                      "or python -m paper_2407_09543_gb300.build (no CPU fallback exists)")
lib = ctypes.CDLL(library_path)


class NTBCError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


c_int, c_size_t, c_void_p, c_float = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_float


class ModelDesc(ctypes.Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("n_textures", c_int), ("formats", c_int * MAX_TEXTURES),
                ("color_levels", c_int), ("color_res", c_int * MAX_LEVELS), ("endpoint_levels", c_int),
                ("endpoint_res", c_int * MAX_LEVELS), ("features", c_int), ("hidden_layers", c_int),
                ("hidden_width", c_int), ("activation", c_int)]

    @classmethod
    def make(cls, width, height, formats, color_res, endpoint_res, hidden_layers=3, activation=ACT_SELU,
             features=2, hidden_width=64):
        d = cls()
        d.width, d.height, d.n_textures = width, height, len(formats)
        for i, f in enumerate(formats):
            d.formats[i] = f
        d.color_levels = len(color_res)
        for i, r in enumerate(color_res):
            d.color_res[i] = r
        d.endpoint_levels = len(endpoint_res)
        for i, r in enumerate(endpoint_res):
            d.endpoint_res[i] = r
        d.features, d.hidden_layers, d.hidden_width, d.activation = features, hidden_layers, hidden_width, activation
        return d


class Span(ctypes.Structure):
    _fields_ = [("offset", c_size_t), ("count", c_size_t)]


class Layout(ctypes.Structure):
    _fields_ = [("total", c_size_t), ("color_grid", Span * MAX_LEVELS), ("endpoint_grid", Span * MAX_LEVELS),
                ("color_w", Span * MAX_MLP_LAYERS), ("color_b", Span * MAX_MLP_LAYERS),
                ("endpoint_w", Span * MAX_MLP_LAYERS), ("endpoint_b", Span * MAX_MLP_LAYERS),
                ("in_color", c_int), ("out_color", c_int), ("in_endpoint", c_int), ("out_endpoint", c_int),
                ("grid_floats", c_size_t)]


class Material(ctypes.Structure):
    _fields_ = [("width", c_int), ("height", c_int), ("n_textures", c_int), ("formats", c_int * MAX_TEXTURES),
                ("texels", c_void_p * MAX_TEXTURES), ("ref_blocks", c_void_p * MAX_TEXTURES)]

    @classmethod
    def make(cls, width, height, formats, texels, ref_blocks):
        m = cls()
        m.width, m.height, m.n_textures = width, height, len(formats)
        for i, f in enumerate(formats):
            m.formats[i] = f
            m.texels[i] = _ptr(texels[i])
            m.ref_blocks[i] = _ptr(ref_blocks[i])
        return m


class TrainConfig(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_long), ("batch_texels", c_int), ("qat_fraction", c_float), ("grid_bits", c_int),
                ("lr_grid", c_float), ("lr_mlp", c_float), ("temperature", c_float), ("warmup", c_int),
                ("seed", ctypes.c_uint64), ("precision", c_int)]

    @classmethod
    def make(cls, steps, batch_texels, qat_fraction=0.0, grid_bits=8, lr_grid=0.01, lr_mlp=0.005,
             temperature=0.01, warmup=10, seed=0, precision=0):
        return cls(steps, batch_texels, qat_fraction, grid_bits, lr_grid, lr_mlp, temperature, warmup, seed, precision)


_P = c_void_p
_SIGS = {
    "ntbc_last_error": (ctypes.c_char_p, []),
    "ntbc_abi_version": (c_int, []),
    "bc_reference_encode": (c_int, [c_int, _P, c_int, c_int, _P, _P]),
    "bc_decode": (c_int, [c_int, _P, c_int, c_int, _P, _P]),
    "bc_reference_encode_refined": (c_int, [c_int, _P, c_int, c_int, c_int, _P, _P]),
    "ntbc_outputs_to_bc": (c_int, [c_int, _P, _P, c_int, _P, _P]),
    "ntbc_model_layout": (c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(Layout)]),
    "ntbc_level_resolutions": (c_int, [c_int, c_int, c_int, ctypes.POINTER(c_int)]),
    "ntbc_model_create": (c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(_P)]),
    "ntbc_model_free": (None, [_P]),
    "ntbc_model_params": (c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(c_size_t)]),
    "ntbc_model_set_params": (c_int, [_P, _P, c_size_t, _P]),
    "ntbc_model_get_params": (c_int, [_P, _P, c_size_t, _P]),
    "ntbc_model_export": (c_int, [_P, c_int, c_int, _P]),
    "ntbc_model_exported_grid": (c_int, [_P, _P, _P, _P, _P]),
    "ntbc_model_blob_size": (c_int, [_P, ctypes.POINTER(c_size_t)]),
    "ntbc_model_save": (c_int, [_P, _P, c_size_t, _P]),
    "ntbc_model_load": (c_int, [_P, _P, c_size_t, _P]),
    "ntbc_infer_to_bc": (c_int, [_P, ctypes.POINTER(_P), _P]),
    "ntbc_forward": (c_int, [_P, _P, c_int, _P, _P, _P]),
    "ntbc_infer_to_bc_strided": (c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(c_int), _P]),
    "ntbc_infer_to_host": (c_int, [_P, ctypes.POINTER(_P), c_int, _P]),
    "ntbc_wait_probe": (c_int, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), _P]),
    "ntbc_train_range": (c_int, [_P, ctypes.POINTER(Material), ctypes.POINTER(TrainConfig), ctypes.c_long,
                                 ctypes.c_long, _P, _P]),
    "ntbc_checkpoint_size": (c_int, [_P, ctypes.POINTER(c_size_t)]),
    "ntbc_checkpoint_save": (c_int, [_P, _P, c_size_t, _P]),
    "ntbc_checkpoint_load": (c_int, [_P, _P, c_size_t, ctypes.POINTER(ctypes.c_long), _P]),
    "ntbc_ex2_rate_probe": (c_int, [ctypes.POINTER(ctypes.c_double), _P]),
    "ntbc_train_grads": (c_int, [_P, ctypes.POINTER(Material), _P, c_int, c_int, c_float, c_int, _P, _P, _P]),
    "ntbc_train_grads_noalloc": (c_int, [ctypes.POINTER(ModelDesc), _P, ctypes.POINTER(Material), _P, c_int, c_int,
                                         c_float, _P, _P, _P]),
    "ntbc_vjp": (c_int, [_P, _P, c_int, c_int, _P, _P, _P, _P, _P, _P]),
    "ntbc_adam_step": (c_int, [_P, _P, ctypes.c_long, ctypes.c_long, ctypes.POINTER(TrainConfig), _P]),
    "ntbc_sample_blocks": (c_int, [ctypes.c_uint64, ctypes.c_long, c_int, c_int, _P, _P]),
    "ntbc_infer_plan": (c_int, [_P, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "ntbc_batch_create": (c_int, [ctypes.POINTER(_P), c_int, ctypes.POINTER(ctypes.POINTER(_P)), ctypes.POINTER(_P)]),
    "ntbc_batch_create_mode": (c_int, [ctypes.POINTER(_P), c_int, ctypes.POINTER(ctypes.POINTER(_P)), c_int,
                                       ctypes.POINTER(_P)]),
    "ntbc_batch_infer": (c_int, [_P, _P]),
    "ntbc_batch_times": (c_int, [_P, ctypes.POINTER(ctypes.c_double), _P]),
    "ntbc_batch_free": (None, [_P]),
    "ntbc_train": (c_int, [_P, ctypes.POINTER(Material), ctypes.POINTER(TrainConfig), ctypes.POINTER(c_float), _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status):
    if status != 0:
        raise NTBCError(status, lib.ntbc_last_error().decode())


def _ptr(t):
    """Device (or host) address of a tensor / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    return stream if isinstance(stream, int) else stream.cuda_stream


def bc_reference_encode(fmt, texels, w, h, blocks, stream=None, refine=0):
    """Reference BC encode; refine > 0 adds that many least-squares refinement steps."""
    if refine:
        _check(lib.bc_reference_encode_refined(fmt, _ptr(texels), w, h, refine, _ptr(blocks), _stream(stream)))
    else:
        _check(lib.bc_reference_encode(fmt, _ptr(texels), w, h, _ptr(blocks), _stream(stream)))


def bc_decode(fmt, blocks, w, h, texels, stream=None):
    _check(lib.bc_decode(fmt, _ptr(blocks), w, h, _ptr(texels), _stream(stream)))


def ntbc_outputs_to_bc(fmt, e_hat, c_hat, n, blocks, stream=None):
    _check(lib.ntbc_outputs_to_bc(fmt, _ptr(e_hat), _ptr(c_hat), n, _ptr(blocks), _stream(stream)))


def ntbc_level_resolutions(levels, n_min, n_max):
    out = (c_int * levels)()
    _check(lib.ntbc_level_resolutions(levels, n_min, n_max, out))
    return list(out)


def ntbc_model_layout(desc: ModelDesc) -> Layout:
    lay = Layout()
    _check(lib.ntbc_model_layout(ctypes.byref(desc), ctypes.byref(lay)))
    return lay


def ntbc_sample_blocks(seed, step, n, n_blocks, ids, stream=None):
    _check(lib.ntbc_sample_blocks(seed, step, n, n_blocks, _ptr(ids), _stream(stream)))


def ntbc_wait_probe(polls, stream=None):
    """Bounded-wait failure path: returns (status, seconds); NTBC_ETIMEOUT (4) is the expected
    status (the wait on an mbarrier that nothing completes gave up)."""
    sec = ctypes.c_double(0.0)
    status = lib.ntbc_wait_probe(polls, ctypes.byref(sec), _stream(stream))
    return status, sec.value


def ntbc_ex2_rate_probe(stream=None):
    """exp2 results per second of the whole device (the MUFU peak of the inference roofline)."""
    rate = ctypes.c_double(0.0)
    _check(lib.ntbc_ex2_rate_probe(ctypes.byref(rate), _stream(stream)))
    return rate.value


NOALLOC_MAX_BLOCKS = 128


def ntbc_train_grads_noalloc(desc: ModelDesc, params, material: Material, block_ids, grads, losses, qat_bits=0,
                             temperature=0.01, stream=None):
    """Allocation-free ntbc_train_grads on caller-owned FP32 parameters (see include/ntbc.h)."""
    _check(lib.ntbc_train_grads_noalloc(ctypes.byref(desc), _ptr(params), ctypes.byref(material), _ptr(block_ids),
                                        block_ids.numel(), qat_bits, temperature, _ptr(grads), _ptr(losses),
                                        _stream(stream)))


class Model:
    """Owner of one opaque ntbc_model handle (library-owned device state)."""

    def __init__(self, desc: ModelDesc):
        self.desc = desc
        self.layout = ntbc_model_layout(desc)
        h = _P()
        _check(lib.ntbc_model_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib.ntbc_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_params(self):
        return self.layout.total

    def set_params(self, flat, stream=None):
        _check(lib.ntbc_model_set_params(self.handle, _ptr(flat), flat.numel(), _stream(stream)))

    def get_params(self, out, stream=None):
        _check(lib.ntbc_model_get_params(self.handle, _ptr(out), out.numel(), _stream(stream)))

    def export(self, grid_bits=8, weight_prec=PREC_FP16, stream=None):
        _check(lib.ntbc_model_export(self.handle, grid_bits, weight_prec, _stream(stream)))

    def exported_grid(self, codes, scales, zeros, stream=None):
        _check(lib.ntbc_model_exported_grid(self.handle, _ptr(codes), _ptr(scales), _ptr(zeros), _stream(stream)))

    def blob_size(self):
        n = c_size_t()
        _check(lib.ntbc_model_blob_size(self.handle, ctypes.byref(n)))
        return n.value

    def save(self, host_buf, stream=None):
        _check(lib.ntbc_model_save(self.handle, _ptr(host_buf), host_buf.numel(), _stream(stream)))

    def load(self, host_buf, stream=None):
        _check(lib.ntbc_model_load(self.handle, _ptr(host_buf), host_buf.numel(), _stream(stream)))

    def infer_to_bc(self, blocks_out, stream=None, strides=None):
        """blocks_out: per texture a device tensor (or an int address) of its first block;
        strides: optional bytes between blocks per texture (8 or 16; BC3 / BC5 layouts)."""
        arr = (_P * len(blocks_out))(*[_ptr(b) for b in blocks_out])
        if strides is None:
            _check(lib.ntbc_infer_to_bc(self.handle, arr, _stream(stream)))
        else:
            st = (c_int * len(strides))(*strides)
            _check(lib.ntbc_infer_to_bc_strided(self.handle, arr, st, _stream(stream)))

    def infer_to_host(self, host_out, chunks=4, stream=None):
        """host_out: per texture a host tensor (pinned for overlap) or int address of its first
        block; the blocks are there once the stream has been synchronised."""
        arr = (_P * len(host_out))(*[_ptr(b) for b in host_out])
        _check(lib.ntbc_infer_to_host(self.handle, arr, chunks, _stream(stream)))

    def infer_plan(self):
        """(kernel launches per infer_to_bc call, blocks per work unit, work units in flight)."""
        l, u, f = c_int(), c_int(), c_int()
        _check(lib.ntbc_infer_plan(self.handle, ctypes.byref(l), ctypes.byref(u), ctypes.byref(f)))
        return l.value, u.value, f.value

    def forward(self, block_ids, e_hat, c_hat, stream=None):
        _check(lib.ntbc_forward(self.handle, _ptr(block_ids), block_ids.numel(), _ptr(e_hat), _ptr(c_hat),
                                _stream(stream)))

    def train_grads(self, material: Material, block_ids, grads, losses=None, qat_bits=0, temperature=0.01,
                    precision=0, stream=None):
        _check(lib.ntbc_train_grads(self.handle, ctypes.byref(material), _ptr(block_ids), block_ids.numel(),
                                    qat_bits, temperature, precision, _ptr(grads), _ptr(losses), _stream(stream)))

    def vjp(self, block_ids, qat_bits=0, g_e=None, g_c=None, grads=None, e_hat=None, c_hat=None, stream=None):
        _check(lib.ntbc_vjp(self.handle, _ptr(block_ids), block_ids.numel(), qat_bits, _ptr(g_e), _ptr(g_c),
                            _ptr(grads), _ptr(e_hat), _ptr(c_hat), _stream(stream)))

    def adam_step(self, grads, step, total_steps, cfg: TrainConfig, stream=None):
        _check(lib.ntbc_adam_step(self.handle, _ptr(grads), step, total_steps, ctypes.byref(cfg), _stream(stream)))

    def train(self, material: Material, cfg: TrainConfig, stream=None):
        out = (c_float * 6)()
        _check(lib.ntbc_train(self.handle, ctypes.byref(material), ctypes.byref(cfg), out, _stream(stream)))
        return list(out)

    def train_range(self, material: Material, cfg: TrainConfig, first_step, last_step, stream=None):
        out = (c_float * 6)()
        _check(lib.ntbc_train_range(self.handle, ctypes.byref(material), ctypes.byref(cfg), first_step, last_step, out,
                                    _stream(stream)))
        return list(out)

    def checkpoint_size(self):
        n = c_size_t()
        _check(lib.ntbc_checkpoint_size(self.handle, ctypes.byref(n)))
        return n.value

    def checkpoint_save(self, host_buf, stream=None):
        _check(lib.ntbc_checkpoint_save(self.handle, _ptr(host_buf), host_buf.numel(), _stream(stream)))

    def checkpoint_load(self, host_buf, stream=None):
        """Returns the step a resumed encode starts at."""
        step = ctypes.c_long(0)
        _check(lib.ntbc_checkpoint_load(self.handle, _ptr(host_buf), host_buf.numel(), ctypes.byref(step),
                                        _stream(stream)))
        return step.value


class Batch:
    """Many materials (each its own exported Model) decoded to BC blocks by one call: chained
    single-material launches (BATCH_CHAINED, the default) or one persistent work-queue launch
    (BATCH_QUEUE)."""

    def __init__(self, models, blocks_out, mode=None):
        self.models = list(models)
        self.n = len(self.models)
        self._outs = [(_P * len(o))(*[_ptr(b) for b in o]) for o in blocks_out]
        outer = (ctypes.POINTER(_P) * self.n)(*[ctypes.cast(o, ctypes.POINTER(_P)) for o in self._outs])
        handles = (_P * self.n)(*[m.handle for m in self.models])
        h = _P()
        if mode is None:
            _check(lib.ntbc_batch_create(handles, self.n, outer, ctypes.byref(h)))
        else:
            _check(lib.ntbc_batch_create_mode(handles, self.n, outer, mode, ctypes.byref(h)))
        self.handle = h

    def infer(self, stream=None):
        _check(lib.ntbc_batch_infer(self.handle, _stream(stream)))

    def times_ms(self, stream=None):
        out = (ctypes.c_double * self.n)()
        _check(lib.ntbc_batch_times(self.handle, out, _stream(stream)))
        return list(out)

    def close(self):
        if getattr(self, "handle", None):
            lib.ntbc_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

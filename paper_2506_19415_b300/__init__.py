"""Python binding of libvm3dgs (virtual-memory 3D Gaussian Splatting on one GPU).

Argument marshalling only: every step of the per-frame path runs in the CUDA
kernels of ``libvm3dgs.so``; PyTorch supplies device memory (the page pool,
the scratch area, the images) and streams.  The functions carry the names of
the C ABI declared in ``include/vm3dgs.h``.  Importing this package fails
loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvm3dgs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libvm3dgs.so is not built; run `python paper_2506_19415_b300/_build.py` "
                      "(or __graft_entry__.build()) first")
_lib = ctypes.CDLL(LIB_PATH)

OK, E_INVAL, E_CAPACITY, E_CUDA, E_TIMEOUT, E_STATE, E_NOMEM = 0, -1, -2, -3, -4, -5, -6


class Vm3dgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("vm3dgs error %d: %s" % (code, msg))
        self.code = code


c_f, c_i32, c_i64, c_u64, c_d, c_p = ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class Gaussians(ctypes.Structure):
    _fields_ = [("n", c_i64), ("sh_degree", c_i32), ("pos", c_p), ("log_scale", c_p), ("rot", c_p),
                ("op_logit", c_p), ("f_dc", c_p), ("f_rest", c_p)]


class BuildParams(ctypes.Structure):
    _fields_ = [("page_size", c_i32), ("paging", c_i32), ("lod_levels", c_i32), ("lod_fanout", c_i32),
                ("lo", c_d * 3), ("hi", c_d * 3), ("voxel", c_d), ("kappa", c_d), ("closing", c_i32),
                ("link_samples", c_i32), ("link_sigma", c_d), ("seed", c_u64), ("links", c_i32), ("fp16", c_i32),
                ("n_threads", c_i32), ("lod_method", c_i32), ("kmeans_iters", c_i32), ("kmeans_scale", c_d),
                ("kmeans_attr_weight", c_d), ("mesh_kappa", c_d), ("mesh_op_min", c_d), ("mesh_closing", c_i32),
                ("mesh_qem_ratio", c_d)]


class Camera(ctypes.Structure):
    _fields_ = [("view", c_f * 12), ("campos", c_f * 3), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("width", c_i32), ("height", c_i32), ("tile_w", c_i32), ("tile_h", c_i32)]


class Params(ctypes.Structure):
    _fields_ = [("staging_bytes", c_i64), ("feedback_ds", c_i32), ("links", c_i32), ("lod", c_i32),
                ("fp16_pool", c_i32), ("usage_lo", c_f), ("usage_hi", c_f), ("tau0", c_f), ("step0", c_f),
                ("max_width", c_i32), ("max_height", c_i32), ("max_views", c_i32), ("max_pairs", c_i64),
                ("bg", c_f * 3), ("separate_values", c_i32), ("sort_mode", c_i32), ("lod_fade_frames", c_i32)]


class Stats(ctypes.Structure):
    _fields_ = [("frame", c_i32), ("requested", c_i32), ("direct", c_i32), ("resident", c_i32), ("missing", c_i32),
                ("streamed_pages", c_i32), ("streamed_bytes", c_i64), ("drawn_pages", c_i32),
                ("drawn_gaussians", c_i64), ("pairs", c_i64), ("usage", c_f), ("tau", c_f), ("status", c_i32),
                ("acc_frames", c_i64), ("acc_views", c_i64), ("acc_pairs", c_i64), ("acc_drawn_gaussians", c_i64),
                ("acc_streamed_bytes", c_i64), ("acc_streamed_pages", c_i64), ("acc_missing", c_i64),
                ("acc_requested", c_i64), ("acc_prefetched_pages", c_i64), ("acc_prefetched_bytes", c_i64),
                ("acc_prefetch_hits", c_i64), ("staged_projection", c_i32), ("key_tile_bits", c_i32),
                ("key_depth_bits", c_i32), ("key_index_bits", c_i32), ("key_packed", c_i32), ("fading", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SceneInfo(ctypes.Structure):
    _fields_ = [("n_pages", c_i32), ("page_size", c_i32), ("lod_levels", c_i32), ("lod_fanout", c_i32),
                ("sh_degree", c_i32), ("n_gaussians", c_i64), ("record_bytes", c_i32), ("record_bytes16", c_i32),
                ("n_tris", c_i64), ("n_verts", c_i64), ("n_links", c_i64), ("host_bytes", c_i64),
                ("record_bytes_vq", c_i32), ("n_codes", c_i32)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("n_pages", c_i32), ("page_size", c_i32), ("lod_levels", c_i32), ("lod_fanout", c_i32),
                ("sh_degree", c_i32), ("fp16", c_i32), ("pos", ctypes.POINTER(c_p)), ("scale", ctypes.POINTER(c_p)),
                ("rot", ctypes.POINTER(c_p)), ("opacity", ctypes.POINTER(c_p)), ("sh", ctypes.POINTER(c_p)),
                ("err", c_p), ("count", c_p), ("n_verts", c_i64), ("n_tris", c_i64), ("n_links", c_i64),
                ("verts", c_p), ("tris", c_p), ("face_page", c_p), ("link_ptr", c_p), ("link_col", c_p)]


class MlpConfig(ctypes.Structure):
    _fields_ = [("n_in", c_i32), ("n_hidden", c_i32), ("n_out", c_i32), ("max_batch", c_i32), ("seed", c_u64),
                ("lr", c_f), ("beta1", c_f), ("beta2", c_f), ("eps", c_f)]


_SIGS = {
    "vm3dgs_build_pages": [ctypes.POINTER(Gaussians), ctypes.POINTER(BuildParams), ctypes.POINTER(c_p)],
    "vm3dgs_scene_import": [ctypes.POINTER(SceneDesc), ctypes.POINTER(c_p)],
    "vm3dgs_scene_info_get": [c_p, ctypes.POINTER(SceneInfo)],
    "vm3dgs_scene_export": [c_p, c_i32, c_i32, c_p, c_i64, ctypes.POINTER(c_i64)],
    "vm3dgs_scene_destroy": [c_p],
    "vm3dgs_scene_save": [c_p, ctypes.c_char_p],
    "vm3dgs_scene_open": [ctypes.c_char_p, ctypes.POINTER(c_p)],
    "vm3dgs_scene_quantize_sh": [c_p, c_i32, c_i32, c_i64],
    "vm3dgs_pool_slot_bytes": [c_p, c_i32, ctypes.POINTER(c_i64)],
    "vm3dgs_scratch_bytes": [c_p, ctypes.POINTER(Params), c_i64, ctypes.POINTER(c_i64)],
    "vm3dgs_renderer_create": [c_p, ctypes.POINTER(Params), c_p, c_i64, c_p, c_i64, c_p, ctypes.POINTER(c_p)],
    "vm3dgs_renderer_destroy": [c_p],
    "vm3dgs_render_feedback": [c_p, ctypes.POINTER(Camera), c_i32, c_p],
    "vm3dgs_request_all": [c_p, c_p],
    "vm3dgs_update_residency": [c_p, c_p, c_p],
    "vm3dgs_render": [c_p, ctypes.POINTER(Camera), c_i32, ctypes.POINTER(c_p), c_p],
    "vm3dgs_get_stats": [c_p, ctypes.POINTER(Stats), c_p],
    "vm3dgs_reset_sums": [c_p, c_p],
    "vm3dgs_debug_read": [c_p, c_i32, c_p, c_i64, ctypes.POINTER(c_i64), c_p],
    "vm3dgs_timing_enable": [c_p, c_i32],
    "vm3dgs_timing_read": [c_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_i64), c_i32],
    "vm3dgs_prefetcher_bytes": [ctypes.POINTER(MlpConfig), ctypes.POINTER(c_i64)],
    "vm3dgs_prefetcher_create": [ctypes.POINTER(MlpConfig), c_p, c_i64, c_p, ctypes.POINTER(c_p)],
    "vm3dgs_prefetcher_destroy": [c_p],
    "vm3dgs_prefetcher_forward": [c_p, c_p, c_i32, c_p, c_p],
    "vm3dgs_prefetcher_train_step": [c_p, c_p, c_p, c_p, c_i32, c_f, c_p, c_p],
    "vm3dgs_prefetcher_params": [c_p, c_i32, c_p, c_i64, c_p],
    "vm3dgs_prefetch_features": [c_p, c_i32, ctypes.POINTER(Camera), ctypes.POINTER(Camera), c_p, c_p, c_p],
    "vm3dgs_prefetch_labels": [c_p, c_i32, c_p, c_p, c_p, c_i32, c_p],
    "vm3dgs_prefetch": [c_p, c_p, ctypes.POINTER(Camera), ctypes.POINTER(Camera), c_f, c_p, c_p],
    "vm3dgs_sort_pairs_noalloc": [c_p, c_p, c_i64, c_i32, c_p, c_p],
    "vm3dgs_render_batched": [c_p, ctypes.POINTER(Camera), c_i32, ctypes.POINTER(c_p), c_p],
    "vm3dgs_batch_graph_capture": [c_p, ctypes.POINTER(Camera), c_i32, ctypes.POINTER(c_p), c_p],
    "vm3dgs_batch_graph_launch": [c_p, ctypes.POINTER(Camera), c_i32, c_p],
    "vm3dgs_autotune_tiles": [c_p, ctypes.POINTER(Camera), c_i32, ctypes.POINTER(c_p), c_i32, c_p],
    "vm3dgs_mesh_simplify": [c_p, c_i64, c_p, c_i64, c_i64, c_p, c_p],
    "vm3dgs_mesh_assign_pages": [c_i64, c_p, c_i64, c_p, c_i64, c_p, c_i64, c_i64, c_p, c_i64, c_p, c_p, c_p, c_p,
                                 c_p, c_p],
    "vm3dgs_last_error": [],
    "vm3dgs_version": [],
}
for _n, _a in _SIGS.items():
    _f = getattr(_lib, _n)
    _f.argtypes = _a
    _f.restype = ctypes.c_char_p if _n in ("vm3dgs_last_error", "vm3dgs_version") else (
        None if _n.endswith("destroy") else ctypes.c_int)

EXPORTED = tuple(_SIGS)

# scene export / debug items (mirror the enums of include/vm3dgs.h)
SCENE_PAGE_COUNT, SCENE_PAGE_SRC, SCENE_PAGES, SCENE_PAGES16, SCENE_ERR, SCENE_VERTS, SCENE_TRIS, \
    SCENE_FACE_PAGE, SCENE_LINK_PTR, SCENE_LINK_COL, SCENE_CODEBOOK, SCENE_PAGES_VQ = range(12)
# pool record formats (RenderConfig.fp16_pool; True / False stand for 1 / 0)
POOL_FP32, POOL_FP16, POOL_VQ = 0, 1, 2
(DBG_FEEDBACK, DBG_REQ, DBG_DIRECT, DBG_REQUESTS, DBG_PT_LOD, DBG_PT_LAST, DBG_PT_SLOT, DBG_COPIES, DBG_DRAW,
 DBG_MISSING, DBG_SPLAT_RECT, DBG_SPLAT_DEPTH, DBG_SPLAT_RADIUS, DBG_KEYS, DBG_VALUES, DBG_RANGES, DBG_SPLAT_XY,
 DBG_SPLAT_CONIC, DBG_SPLAT_RGB, DBG_POOL, DBG_RASTER, DBG_SPLAT_TMASK, DBG_SPLAT_TOUCHED, DBG_DRAW_W) = range(24)


STAGES = ("feedback", "residency", "stream", "project", "scan_emit", "sort", "ranges", "blend", "prefetch", "sort_prep")
N_STAGES = len(STAGES)


def _check(rc):
    if rc != OK:
        raise Vm3dgsError(rc, _lib.vm3dgs_last_error().decode())


def version() -> str:
    return _lib.vm3dgs_version().decode()


def _ptr(a):
    return a.ctypes.data_as(c_p) if a is not None else None


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return c_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def camera_struct(cam) -> Camera:
    c = Camera()
    c.view[:] = [float(v) for v in np.asarray(cam.view, np.float32).reshape(-1)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.tile_w, c.tile_h = int(cam.width), int(cam.height), int(cam.tile_w), int(cam.tile_h)
    return c


def camera_array(cams):
    arr = (Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


# --------------------------------------------------------------------------- scene
@dataclass
class BuildConfig:
    page_size: int = 256
    paging: str = "morton"       # or "octree", or "mesh" (the paper's mesh proxy, Sec. 3.1-3.2; needs a GPU)
    lod_levels: int = 1
    lod_fanout: int = 8
    lo: tuple = (-5.0, -5.0, -5.0)
    hi: tuple = (5.0, 5.0, 5.0)
    voxel: float = 10.0 / 32
    kappa: float = 0.5
    closing: bool = True
    link_samples: int = 8
    link_sigma: float = 2.0
    seed: int = 77
    links: bool = True
    fp16: bool = False
    n_threads: int = 0
    lod_method: str = "moment"   # or "kmeans" (Sec. 3.4)
    kmeans_iters: int = 10
    kmeans_scale: float = 0.0    # 0: lod_fanout^(1/3)
    kmeans_attr_weight: float = 0.1
    mesh_kappa: float = 2.0      # paging "mesh": ellipsoid of mesh_kappa sigma
    mesh_op_min: float = 0.1     # Gaussians below this opacity do not occupy
    mesh_closing: int = 1        # closing radius in voxels
    mesh_qem_ratio: float = 0.25 # triangles kept by the simplification

    def struct(self) -> BuildParams:
        b = BuildParams()
        if self.paging not in ("morton", "octree", "mesh"):
            raise ValueError("paging is 'morton', 'octree' or 'mesh'")
        b.page_size, b.paging = self.page_size, {"morton": 0, "octree": 1, "mesh": 2}[self.paging]
        b.mesh_kappa, b.mesh_op_min, b.mesh_closing = self.mesh_kappa, self.mesh_op_min, self.mesh_closing
        b.mesh_qem_ratio = self.mesh_qem_ratio
        b.lod_levels, b.lod_fanout = self.lod_levels, self.lod_fanout
        b.lo[:] = [float(v) for v in self.lo]
        b.hi[:] = [float(v) for v in self.hi]
        b.voxel, b.kappa, b.closing = self.voxel, self.kappa, int(self.closing)
        b.link_samples, b.link_sigma, b.seed = self.link_samples, self.link_sigma, self.seed
        b.links, b.fp16, b.n_threads = int(self.links), int(self.fp16), self.n_threads
        if self.lod_method not in ("moment", "kmeans"):
            raise ValueError("lod_method is 'moment' or 'kmeans'")
        b.lod_method = 1 if self.lod_method == "kmeans" else 0
        b.kmeans_iters, b.kmeans_scale, b.kmeans_attr_weight = self.kmeans_iters, self.kmeans_scale, \
            self.kmeans_attr_weight
        return b


class Scene:
    """Owns a vm3dgs_scene handle."""

    def __init__(self, handle):
        self.h = c_p(handle) if not isinstance(handle, c_p) else handle
        inf = SceneInfo()
        _check(_lib.vm3dgs_scene_info_get(self.h, ctypes.byref(inf)))
        self.info = inf

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.vm3dgs_scene_destroy(self.h)
            self.h = None

    def save(self, path):
        """Writes the scene to a file that vm3dgs_scene_open maps (Sec. 3.5)."""
        _check(_lib.vm3dgs_scene_save(self.h, os.fsencode(path)))

    def export(self, what, level=0, dtype=np.uint8):
        need = c_i64()
        _check(_lib.vm3dgs_scene_export(self.h, what, level, None, 0, ctypes.byref(need)))
        buf = np.empty(need.value, np.uint8)
        _check(_lib.vm3dgs_scene_export(self.h, what, level, _ptr(buf), need.value, ctypes.byref(need)))
        return buf.view(dtype)

    def m(self, l):
        return self.info.page_size // self.info.lod_fanout ** l

    def quantize_sh(self, n_codes, iters=10, n_train=65536):
        """Adds the SH codebook and the VQ page records (compressed pages,
        pool format POOL_VQ); the scene must not have them yet."""
        _check(_lib.vm3dgs_scene_quantize_sh(self.h, int(n_codes), int(iters), int(n_train)))
        inf = SceneInfo()
        _check(_lib.vm3dgs_scene_info_get(self.h, ctypes.byref(inf)))
        self.info = inf

    def codebook(self):
        """The SH codebook as [n_codes, 3 (K - 1)] float32."""
        return self.export(SCENE_CODEBOOK, 0, np.float32).reshape(self.info.n_codes, -1)

    def vq_codes(self, level=0):
        """The codebook index of every Gaussian of a level, [n_pages, m] int32
        (16-bit row 10 of the VQ record)."""
        m = self.m(level)
        b = self.export(SCENE_PAGES_VQ, level).reshape(self.info.n_pages, -1)
        h = b[:, 16 * m:].copy().view(np.uint16).reshape(self.info.n_pages, 12, m)
        return h[:, 10, :].astype(np.int32)

    def pages(self, level=0, fp16=False):
        """Page blocks of a level as [n_pages, bytes] uint8."""
        b = self.export(SCENE_PAGES16 if fp16 else SCENE_PAGES, level)
        return b.reshape(self.info.n_pages, -1)

    def unpack(self, level=0):
        """Level page blocks as dict of [n_pages, m, ...] fp32 arrays (pos, scale, rot, opacity, sh)."""
        K = (self.info.sh_degree + 1) ** 2
        m = self.m(level)
        f = self.pages(level).view(np.float32).reshape(self.info.n_pages, 11 + 3 * K, m)
        f = np.transpose(f, (0, 2, 1))
        return dict(pos=f[..., 0:3].copy(), scale=f[..., 3:6].copy(), rot=f[..., 6:10].copy(),
                    opacity=f[..., 10].copy(), sh=f[..., 11:].reshape(self.info.n_pages, m, K, 3).copy())


def vm3dgs_build_pages(raw, cfg: BuildConfig) -> Scene:
    """raw: object with pos, log_scale, rot, op_logit, f_dc, f_rest (numpy, float32) and sh_degree."""
    arrs = [np.ascontiguousarray(getattr(raw, k), np.float32) for k in ("pos", "log_scale", "rot", "op_logit", "f_dc")]
    rest = np.ascontiguousarray(raw.f_rest, np.float32) if raw.sh_degree > 0 else None
    g = Gaussians(len(arrs[0]), raw.sh_degree, *[_ptr(a) for a in arrs], _ptr(rest))
    h = c_p()
    b = cfg.struct()
    _check(_lib.vm3dgs_build_pages(ctypes.byref(g), ctypes.byref(b), ctypes.byref(h)))
    return Scene(h)


def vm3dgs_scene_save(scene, path):
    scene.save(path)


def vm3dgs_scene_open(path) -> Scene:
    """A scene whose page data stays in a read-only mapping of the file."""
    h = c_p()
    _check(_lib.vm3dgs_scene_open(os.fsencode(path), ctypes.byref(h)))
    return Scene(h)


def vm3dgs_scene_import(levels, err, count, verts, tris, face_page, link_ptr, link_col, page_size, fanout, sh_degree,
                        fp16=False) -> Scene:
    """levels: list of dicts of [n_pages, m_l, ...] arrays (pos, scale, rot, opacity, sh)."""
    keep = []

    def c(a, dt):
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return a

    L = len(levels)
    arrs = {k: [c(lv[k], np.float32) for lv in levels] for k in ("pos", "scale", "rot", "opacity", "sh")}
    ptrs = {k: (c_p * L)(*[v.ctypes.data for v in arrs[k]]) for k in arrs}
    d = SceneDesc()
    d.n_pages, d.page_size, d.lod_levels, d.lod_fanout = levels[0]["opacity"].shape[0], page_size, L, fanout
    d.sh_degree, d.fp16 = sh_degree, int(fp16)
    for k in arrs:
        setattr(d, k, ctypes.cast(ptrs[k], ctypes.POINTER(c_p)))
    d.err = _ptr(c(err, np.float32))
    d.count = _ptr(c(count, np.int64))
    vv, tt, fp = c(verts, np.float32), c(tris, np.int32), c(face_page, np.int32)
    lp, lc = c(link_ptr, np.int64), c(link_col if len(link_col) else np.zeros(1), np.int32)
    d.n_verts, d.n_tris, d.n_links = len(vv), len(tt), int(lp[-1])
    d.verts, d.tris, d.face_page, d.link_ptr, d.link_col = _ptr(vv), _ptr(tt), _ptr(fp), _ptr(lp), _ptr(lc)
    h = c_p()
    _check(_lib.vm3dgs_scene_import(ctypes.byref(d), ctypes.byref(h)))
    return Scene(h)


# --------------------------------------------------------------------------- renderer
@dataclass
class RenderConfig:
    staging_bytes: int = 40 * 2048 * 236     # the paper's staging buffer (~18.4 MiB)
    feedback_ds: int = 4
    links: bool = True
    lod: bool = True
    fp16_pool: bool = False
    usage_lo: float = 0.5
    usage_hi: float = 0.8
    tau0: float = 1.0
    step0: float = 0.1
    max_width: int = 1920
    max_height: int = 1080
    max_views: int = 1
    max_pairs: int = 0
    bg: tuple = (0.0, 0.0, 0.0)
    separate_values: bool = False   # True: always sort (key, splat) pairs instead of packed keys
    sort_mode: int = 0              # 0: a onesweep launch per pass; 1: one cooperative launch for all passes
    lod_fade_frames: int = 0        # LOD cross-fade length in frames (0: off)

    def struct(self) -> Params:
        p = Params()
        p.staging_bytes, p.feedback_ds, p.links, p.lod = self.staging_bytes, self.feedback_ds, int(self.links), int(self.lod)
        p.fp16_pool, p.usage_lo, p.usage_hi, p.tau0, p.step0 = int(self.fp16_pool), self.usage_lo, self.usage_hi, self.tau0, self.step0
        p.max_width, p.max_height, p.max_views, p.max_pairs = self.max_width, self.max_height, self.max_views, self.max_pairs
        p.bg[:] = [float(v) for v in self.bg]
        p.separate_values = int(self.separate_values)
        p.sort_mode = int(self.sort_mode)
        p.lod_fade_frames = int(self.lod_fade_frames)
        return p


def vm3dgs_pool_slot_bytes(scene: Scene, fp16_pool=False) -> int:
    out = c_i64()
    _check(_lib.vm3dgs_pool_slot_bytes(scene.h, int(fp16_pool), ctypes.byref(out)))
    return out.value


def vm3dgs_scratch_bytes(scene: Scene, cfg: RenderConfig, pool_bytes: int) -> int:
    out = c_i64()
    p = cfg.struct()
    _check(_lib.vm3dgs_scratch_bytes(scene.h, ctypes.byref(p), pool_bytes, ctypes.byref(out)))
    return out.value


class Renderer:
    """A renderer over torch-allocated device memory (pool + scratch)."""

    def __init__(self, scene: Scene, cfg: RenderConfig, pool_slots=None, pool_bytes=None, device="cuda"):
        import torch
        self.scene, self.cfg = scene, cfg
        slot = vm3dgs_pool_slot_bytes(scene, cfg.fp16_pool)
        if pool_bytes is None:
            pool_bytes = slot * (pool_slots if pool_slots is not None else scene.info.n_pages)
        self.slot_bytes = slot
        self.pool = torch.empty(max(int(pool_bytes), 1), dtype=torch.uint8, device=device)
        sb = vm3dgs_scratch_bytes(scene, cfg, int(pool_bytes))
        self.scratch = torch.empty(sb, dtype=torch.uint8, device=device)
        self.p = cfg.struct()
        self.h = c_p()
        _check(_lib.vm3dgs_renderer_create(scene.h, ctypes.byref(self.p), c_p(self.pool.data_ptr()), int(pool_bytes),
                                           c_p(self.scratch.data_ptr()), sb, _stream_ptr(None), ctypes.byref(self.h)))
        self.n_slots = int(pool_bytes) // slot

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.vm3dgs_renderer_destroy(self.h)
            self.h = None

    def render_feedback(self, cams, stream=None):
        arr = camera_array(cams)
        _check(_lib.vm3dgs_render_feedback(self.h, arr, len(cams), _stream_ptr(stream)))

    def request_all(self, stream=None):
        _check(_lib.vm3dgs_request_all(self.h, _stream_ptr(stream)))

    def update_residency(self, stream=None, copy_stream=None):
        _check(_lib.vm3dgs_update_residency(self.h, _stream_ptr(stream),
                                            _stream_ptr(copy_stream) if copy_stream is not None else None))

    def render(self, cams, images=None, stream=None):
        import torch
        if images is None:
            images = [torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.pool.device) for c in cams]
        arr = camera_array(cams)
        ptrs = (c_p * len(images))(*[im.data_ptr() for im in images])
        _check(_lib.vm3dgs_render(self.h, arr, len(cams), ptrs, _stream_ptr(stream)))
        return images

    def _images(self, cams, images):
        import torch
        if images is None:
            images = [torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.pool.device) for c in cams]
        return images, (c_p * len(images))(*[im.data_ptr() for im in images])

    def render_batched(self, cams, images=None, stream=None):
        images, ptrs = self._images(cams, images)
        _check(_lib.vm3dgs_render_batched(self.h, camera_array(cams), len(cams), ptrs, _stream_ptr(stream)))
        return images

    def batch_graph_capture(self, cams, images=None, stream=None):
        images, ptrs = self._images(cams, images)
        _check(_lib.vm3dgs_batch_graph_capture(self.h, camera_array(cams), len(cams), ptrs, _stream_ptr(stream)))
        return images

    def batch_graph_launch(self, cams, stream=None):
        _check(_lib.vm3dgs_batch_graph_launch(self.h, camera_array(cams), len(cams), _stream_ptr(stream)))

    def autotune_tiles(self, cams, images=None, repeats=3, stream=None):
        """Returns the cameras with the tile shapes the autotuner chose."""
        import copy
        images, ptrs = self._images(cams, images)
        arr = camera_array(cams)
        _check(_lib.vm3dgs_autotune_tiles(self.h, arr, len(cams), ptrs, repeats, _stream_ptr(stream)))
        out = []
        for i, c in enumerate(cams):
            c2 = copy.copy(c)
            c2.tile_w, c2.tile_h = arr[i].tile_w, arr[i].tile_h
            out.append(c2)
        return out

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(_lib.vm3dgs_get_stats(self.h, ctypes.byref(s), _stream_ptr(stream)))
        return s.as_dict()

    def reset_sums(self, stream=None):
        _check(_lib.vm3dgs_reset_sums(self.h, _stream_ptr(stream)))

    def timing(self, on=True):
        _check(_lib.vm3dgs_timing_enable(self.h, int(on)))

    def timing_read(self):
        """(ms per stage, kernel launches per stage) since the last read; synchronises."""
        ms = (ctypes.c_double * N_STAGES)()
        ln = (c_i64 * N_STAGES)()
        _check(_lib.vm3dgs_timing_read(self.h, ms, ln, N_STAGES))
        return list(ms), list(ln)

    def debug(self, what, dtype=np.uint8, stream=None):
        need = c_i64()
        _check(_lib.vm3dgs_debug_read(self.h, what, None, 0, ctypes.byref(need), _stream_ptr(stream)))
        buf = np.empty(max(need.value, 0), np.uint8)
        _check(_lib.vm3dgs_debug_read(self.h, what, _ptr(buf), need.value, ctypes.byref(need), _stream_ptr(stream)))
        return buf.view(dtype)


# thin aliases with the C names
def vm3dgs_renderer_create(scene, cfg, pool_slots=None, pool_bytes=None):
    return Renderer(scene, cfg, pool_slots, pool_bytes)


def vm3dgs_render_feedback(r: Renderer, cams, stream=None):
    r.render_feedback(cams, stream)


def vm3dgs_request_all(r: Renderer, stream=None):
    r.request_all(stream)


def vm3dgs_update_residency(r: Renderer, stream=None, copy_stream=None):
    r.update_residency(stream, copy_stream)


def vm3dgs_render(r: Renderer, cams, images=None, stream=None):
    return r.render(cams, images, stream)


def vm3dgs_get_stats(r: Renderer, stream=None):
    return r.stats(stream)


def vm3dgs_debug_read(r: Renderer, what, dtype=np.uint8, stream=None):
    return r.debug(what, dtype, stream)


# --------------------------------------------------------------------------- prefetcher
PARAMS_GET, PARAMS_SET, PARAMS_GRAD = 0, 1, 2


@dataclass
class MlpShape:
    n_in: int = 12 + 256
    n_hidden: int = 256
    n_out: int = 4096
    max_batch: int = 256
    seed: int = 5
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def struct(self) -> MlpConfig:
        return MlpConfig(self.n_in, self.n_hidden, self.n_out, self.max_batch, self.seed, self.lr, self.beta1,
                         self.beta2, self.eps)


class Prefetcher:
    """The learned page prefetcher over a torch-allocated device buffer."""

    def __init__(self, shape: MlpShape = MlpShape(), device="cuda"):
        import torch
        self.shape = shape
        self.cfg = shape.struct()
        n = c_i64()
        _check(_lib.vm3dgs_prefetcher_bytes(ctypes.byref(self.cfg), ctypes.byref(n)))
        self.mem = torch.empty(n.value, dtype=torch.uint8, device=device)
        self.h = c_p()
        _check(_lib.vm3dgs_prefetcher_create(ctypes.byref(self.cfg), c_p(self.mem.data_ptr()), n.value,
                                             _stream_ptr(None), ctypes.byref(self.h)))
        I, H, O = shape.n_in, shape.n_hidden, shape.n_out
        self.sizes = [("W1", (I, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, O)), ("b3", (O,))]
        self.n_params = sum(int(np.prod(sz)) for _, sz in self.sizes)

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.vm3dgs_prefetcher_destroy(self.h)
            self.h = None

    def _unpack(self, flat):
        out, o = {}, 0
        for k, sz in self.sizes:
            n = int(np.prod(sz))
            out[k] = flat[o:o + n].reshape(sz)
            o += n
        return out

    def params(self):
        buf = np.empty(self.n_params, np.float32)
        _check(_lib.vm3dgs_prefetcher_params(self.h, PARAMS_GET, _ptr(buf), self.n_params, _stream_ptr(None)))
        return self._unpack(buf)

    def grads(self):
        buf = np.empty(self.n_params, np.float32)
        _check(_lib.vm3dgs_prefetcher_params(self.h, PARAMS_GRAD, _ptr(buf), self.n_params, _stream_ptr(None)))
        return self._unpack(buf)

    def set_params(self, P):
        flat = np.concatenate([np.asarray(P[k], np.float32).reshape(-1) for k, _ in self.sizes])
        _check(_lib.vm3dgs_prefetcher_params(self.h, PARAMS_SET, _ptr(flat), self.n_params, _stream_ptr(None)))

    def forward(self, x, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((x.shape[0], self.shape.n_out), dtype=torch.float32, device=x.device)
        _check(_lib.vm3dgs_prefetcher_forward(self.h, c_p(x.data_ptr()), x.shape[0], c_p(out.data_ptr()),
                                              _stream_ptr(stream)))
        return out

    def train_step(self, x, y, mask, loss_out=None, stream=None):
        ms = float(mask.sum().item()) if not hasattr(self, "_fixed_mask_sum") else self._fixed_mask_sum
        _check(_lib.vm3dgs_prefetcher_train_step(self.h, c_p(x.data_ptr()), c_p(y.data_ptr()), c_p(mask.data_ptr()),
                                                 x.shape[0], ms, c_p(loss_out.data_ptr()) if loss_out is not None else None,
                                                 _stream_ptr(stream)))


def vm3dgs_prefetch_features(r: "Renderer", n_out, cam, prev, x_out, base_out=None, stream=None):
    c, pc = camera_struct(cam), camera_struct(prev)
    _check(_lib.vm3dgs_prefetch_features(r.h, n_out, ctypes.byref(c), ctypes.byref(pc), c_p(x_out.data_ptr()),
                                         c_p(base_out.data_ptr()) if base_out is not None else None,
                                         _stream_ptr(stream)))


def vm3dgs_prefetch_labels(r: "Renderer", n_out, base_dev, y_out, mask_out, accumulate=False, stream=None):
    _check(_lib.vm3dgs_prefetch_labels(r.h, n_out, c_p(base_dev.data_ptr()), c_p(y_out.data_ptr()),
                                       c_p(mask_out.data_ptr()), 1 if accumulate else 0, _stream_ptr(stream)))


def vm3dgs_prefetch(r: "Renderer", p: Prefetcher, cam, prev, threshold=0.0, stream=None, copy_stream=None):
    c, pc = camera_struct(cam), camera_struct(prev)
    _check(_lib.vm3dgs_prefetch(r.h, p.h, ctypes.byref(c), ctypes.byref(pc), float(threshold), _stream_ptr(stream),
                                _stream_ptr(copy_stream) if copy_stream is not None else None))


NOALLOC_MAX_PAIRS = 1 << 19


def vm3dgs_sort_pairs_noalloc(keys, vals, n, key_bits, status=None, stream=None):
    """Stable in-place sort of device tensors keys (uint64 as int64) / vals
    (int32) by the low key_bits bits, with the library's fixed scratch (no
    allocation).  status: optional 1-element int32 device tensor.  The
    tensors are checked here (device, layout, dtype, size), since the C ABI
    sees only their addresses."""
    import torch

    def _dev(t, dts, need, what):
        if not (t.is_cuda and t.is_contiguous() and t.dtype in dts):
            raise Vm3dgsError(E_INVAL, "%s must be a contiguous CUDA tensor of dtype %s" % (what, dts))
        if t.numel() < need:
            raise Vm3dgsError(E_INVAL, "%s holds %d elements, fewer than %d" % (what, t.numel(), need))

    n = int(n)
    if 0 <= n <= NOALLOC_MAX_PAIRS:
        _dev(keys, (torch.int64, torch.uint64), n, "keys")
        _dev(vals, (torch.int32, torch.uint32), n, "vals")
    if status is not None:
        _dev(status, (torch.int32,), 1, "status")
    _check(_lib.vm3dgs_sort_pairs_noalloc(c_p(keys.data_ptr()), c_p(vals.data_ptr()), int(n), int(key_bits),
                                          c_p(status.data_ptr()) if status is not None else None,
                                          _stream_ptr(stream)))


# --------------------------------------------------------------------------- mesh proxy host steps
def _np_ptr(a):
    return c_p(a.ctypes.data)


def vm3dgs_mesh_simplify(verts, tris, target):
    """Quadric edge collapses of a mesh (the host step of the mesh proxy);
    returns (verts [nv,3] float64, tris [nt,3] int32)."""
    import numpy as np
    V = np.ascontiguousarray(verts, np.float64).reshape(-1, 3).copy()
    T = np.ascontiguousarray(tris, np.int32).reshape(-1, 3).copy()
    nv, nt = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.vm3dgs_mesh_simplify(_np_ptr(V), len(V), _np_ptr(T), len(T), int(target), ctypes.byref(nv),
                                     ctypes.byref(nt)))
    return V[:nv.value].copy(), T[:nt.value].copy()


def vm3dgs_mesh_assign_pages(mu, page_size, verts, tris):
    """Page assignment by nearest triangle with subdivision and merging (the
    host step of paging "mesh"); returns dict(verts, tris, face_page, order,
    counts)."""
    import numpy as np
    mu = np.ascontiguousarray(mu, np.float32).reshape(-1, 3)
    V = np.ascontiguousarray(verts, np.float64).reshape(-1, 3)
    T = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    n = len(mu)
    cap_v, cap_t = len(V) + 18 * n + 16, len(T) + 18 * n + 16   # splits: at most 17 per mean
    vo = np.zeros((cap_v, 3), np.float64)
    to = np.zeros((cap_t, 3), np.int32)
    fp = np.zeros(cap_t, np.int32)
    order = np.zeros(max(n, 1), np.int64)
    counts = np.zeros(max(n, 1), np.int64)
    parent = np.zeros(max(n, 1), np.int64)
    sizes = np.zeros(3, np.int64)
    _check(_lib.vm3dgs_mesh_assign_pages(n, _np_ptr(mu), int(page_size), _np_ptr(V), len(V), _np_ptr(T), len(T),
                                         cap_v, _np_ptr(vo), cap_t, _np_ptr(to), _np_ptr(fp), _np_ptr(order),
                                         _np_ptr(counts), _np_ptr(parent), _np_ptr(sizes)))
    nv, nt, np_ = (int(x) for x in sizes)
    return dict(verts=vo[:nv].copy(), tris=to[:nt].copy(), face_page=fp[:nt].copy(), order=order[:n].copy(),
                counts=counts[:np_].copy(), parent=parent[:np_].copy())

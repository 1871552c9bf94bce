// C ABI of the warm-start neural operator (include/nop.h): network buffers,
// forward pass, reverse pass, Adam training step and the hand-off of a
// predicted field to a 2D solver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nop.h"
#include "handle.cuh"
#include "nop_kernels.cuh"

using namespace lbmib::nop;
using lbmib_host::DeviceGuard;

namespace {

// one activation tensor: level (resolution H >> level) and channel count
struct Tensor {
  int level, C;
  float* act = nullptr;   // [max_batch][H_l][W_l][C]
  float* grad = nullptr;  // same shape
};

enum OpKind { kConv, kPool, kUp, kAdd };

struct Op {
  OpKind kind;
  int in, in2, out;  // tensor indices (in2: second summand of kAdd)
  int layer;         // conv layer index
  int relu;
};

struct Layer {
  int cin, cout;       // real channel counts
  int cinp, coutp;     // padded to multiples of 16
  long long offset;    // of W in the flat parameter vector (b follows W)
  __nv_bfloat16* Wt = nullptr;
  __nv_bfloat16* Wf = nullptr;
  float* bias = nullptr;
  float* dW = nullptr;  // padded weight gradient [coutp][9][cinp]
  float* db = nullptr;  // padded bias gradient [coutp]
  float* Wt32 = nullptr;  // FP32 weights of the gradient-check mode (nop_set_fp32)
  float* Wf32 = nullptr;
  long long size() const { return (long long)cout * 9 * cin + cout; }
};

int pad16(int c) { return (c + 15) / 16 * 16; }

}  // namespace

struct nop_net {
  nop_config cfg;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<Tensor> T;
  std::vector<Op> ops;
  std::vector<Layer> L;
  int x_t = 0, y_t = 0;   // input and output tensors
  long long n_params = 0;
  float* master = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* part = nullptr;  // weight-gradient chunk partials
  long long part_len = 0;
  double* loss_part = nullptr;
  int loss_blocks = 0;
  double* loss_dev = nullptr;
  double* fields = nullptr;  // rho, u (2 planes), T for nop_infer_into
  long long adam_t = 0;
  bool prepared = false;
  bool fp32 = false;         // FP32 operand convolutions (nop_set_fp32)
  int* tc_status = nullptr;  // set by a tensor-core convolution whose MMA wait timed out
  std::vector<void*> allocs;
};

namespace {

lbm_status fail(nop_net* n, lbm_status s, const std::string& what) {
  n->err = what;
  return s;
}

#define NCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(net, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

long long pixels(const nop_net* net, int level, int batch) {
  return (long long)batch * (net->cfg.height >> level) * (net->cfg.width >> level);
}

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// weight-gradient partials of a level: kWUnits row segments of kRowPx pixels each
int wgrad_chunks(int B, int H, int W) {
  const long long units = (long long)B * H * ((W + kRowPx - 1) / kRowPx);
  return (int)((units + kWUnits - 1) / kWUnits);
}

int add_tensor(nop_net* net, int level, int C) {
  Tensor t;
  t.level = level;
  t.C = C;
  net->T.push_back(t);
  return (int)net->T.size() - 1;
}

int add_conv(nop_net* net, int in, int cin, int cout, int relu) {
  Layer l;
  l.cin = cin;
  l.cout = cout;
  l.cinp = pad16(cin);
  l.coutp = pad16(cout);
  l.offset = net->n_params;
  net->n_params += l.size();
  net->L.push_back(l);
  const int out = add_tensor(net, net->T[in].level, l.coutp);
  net->ops.push_back(Op{kConv, in, -1, out, (int)net->L.size() - 1, relu});
  return out;
}

// The U-Net of include/nop.h, recorded as a list of operations.
void build_graph(nop_net* net) {
  const int* c = net->cfg.channels;
  net->x_t = add_tensor(net, 0, pad16(net->cfg.in_channels));
  int e[4];
  int in = net->x_t, cin = net->cfg.in_channels;
  for (int l = 0; l < 4; ++l) {
    if (l > 0) {
      const int p = add_tensor(net, l, net->T[e[l - 1]].C);
      net->ops.push_back(Op{kPool, e[l - 1], -1, p, -1, 0});
      in = p;
      cin = c[l - 1];
    }
    const int a = add_conv(net, in, cin, c[l], 1);
    e[l] = add_conv(net, a, c[l], c[l], 1);
  }
  int g = e[3];
  for (int l = 2; l >= 0; --l) {
    const int u = add_tensor(net, l, net->T[g].C);
    net->ops.push_back(Op{kUp, g, -1, u, -1, 0});
    const int s = add_conv(net, u, c[l + 1], c[l], 1);
    const int t = add_tensor(net, l, c[l]);
    net->ops.push_back(Op{kAdd, s, e[l], t, -1, 0});
    g = add_conv(net, t, c[l], c[l], 1);
  }
  net->y_t = add_conv(net, g, c[0], net->cfg.out_channels, 0);
}

template <class T>
lbm_status dalloc(nop_net* net, T** p, long long count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (size_t)count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(net, LBM_ENOMEM, "device allocation of the network buffers failed");
  }
  net->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return LBM_OK;
}

lbm_status launch_check(nop_net* net, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(net, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return LBM_OK;
}

// after the stream has been synchronized: launch errors, then the
// tensor-core convolutions' wait status
lbm_status finish(nop_net* net, const char* what) {
  lbm_status s = launch_check(net, what);
  if (s) return s;
  int st = 0;
  if (cudaMemcpy(&st, net->tc_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(net, LBM_ECUDA, std::string(what) + ": status read");
  }
  if (st) {
    cudaMemset(net->tc_status, 0, sizeof(int));
    return fail(net, LBM_ETIMEOUT, std::string(what) + ": a tensor-core convolution timed out waiting for its MMAs");
  }
  return LBM_OK;
}

// the tensor-core convolution with chunks of 8 NG input channels; its
// dynamic shared-memory limit (for the largest Cout, 128) is set once per
// device
template <int NG, bool DB, int R>
void conv_tc(nop_net* net, const float* X, const __nv_bfloat16* Wt, const float* bias, float* Y, int B, int H, int W,
             int Cin, int Cout, int relu, int accumulate) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaFuncSetAttribute(k_conv3x3_tc<NG, DB, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)conv_tc_smem(NG, 128, DB, R));
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  const unsigned grid = (unsigned)((long long)B * (H / R) * (W / kTcM));
  k_conv3x3_tc<NG, DB, R><<<grid, 128 * R, conv_tc_smem(NG, Cout, DB, R), net->st>>>(X, Wt, bias, Y, B, H, W, Cin, Cout,
                                                                                 relu, accumulate, net->tc_status);
}

constexpr int kTcRows = 4;  // image rows per tensor-core CTA (when H allows)

// grid of the row-wise resampling kernels: (x, channel group) of one row
// along x, rows along y (grid-stride beyond 65535 rows)
dim3 row_grid(int rows, int W, int C) {
  return dim3((unsigned)((W * (C / 4) + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
}

// one 3x3 convolution (see k_conv3x3): on the tcgen05 tensor cores when a
// CTA's 128 pixels fit an image row and the output channels one
// accumulator (W % 128 == 0, Cout <= 128), else on the mma.sync path
void conv(nop_net* net, const float* X, const __nv_bfloat16* Wt, const float* bias, float* Y, int B, int H, int W,
          int Cin, int Cout, int relu, int accumulate) {
  if (W % kTcM == 0 && Cout <= 128) {
    if (H % kTcRows == 0) {
      if (Cin % 32 == 0)
        conv_tc<4, false, kTcRows>(net, X, Wt, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
      else
        conv_tc<2, false, kTcRows>(net, X, Wt, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
    } else {
      if (Cin % 32 == 0)
        conv_tc<4, false, 1>(net, X, Wt, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
      else
        conv_tc<2, false, 1>(net, X, Wt, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
    }
    return;
  }
  dim3 grid((unsigned)((long long)B * H * ((W + kRowPx - 1) / kRowPx)), (unsigned)((Cout + kTN - 1) / kTN));
  k_conv3x3<<<grid, 128, 0, net->st>>>(X, Wt, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
}

// the FP32 operand convolution of the gradient-check mode
void conv_f32(nop_net* net, const float* X, const float* W32, const float* bias, float* Y, int B, int H, int W,
              int Cin, int Cout, int relu, int accumulate) {
  const long long n = (long long)B * H * W * Cout;
  k_conv3x3_f32<<<blocks(n), 256, 0, net->st>>>(X, W32, bias, Y, B, H, W, Cin, Cout, relu, accumulate);
}

// BF16 copies of the master weights (after every change of the masters)
lbm_status prepare(nop_net* net) {
  if (net->prepared) return LBM_OK;
  for (Layer& l : net->L) {
    const long long n = (long long)l.coutp * 9 * l.cinp;
    k_prep_layer<<<blocks(n), 256, 0, net->st>>>(net->master + l.offset, l.cin, l.cout, l.cinp, l.coutp, l.Wt,
                                                 l.Wf, l.bias);
    if (net->fp32)
      k_prep_layer_f32<<<blocks(n), 256, 0, net->st>>>(net->master + l.offset, l.cin, l.cout, l.cinp, l.coutp,
                                                       l.Wt32, l.Wf32);
  }
  net->prepared = true;
  return launch_check(net, "k_prep_layer");
}

lbm_status forward(nop_net* net, int B) {
  lbm_status s = prepare(net);
  if (s) return s;
  const int H = net->cfg.height, W = net->cfg.width;
  for (const Op& op : net->ops) {
    const Tensor& ti = net->T[op.in];
    const Tensor& to = net->T[op.out];
    const int Ho = H >> to.level, Wo = W >> to.level;
    const long long n_out = pixels(net, to.level, B) * to.C;
    switch (op.kind) {
      case kConv: {
        const Layer& l = net->L[op.layer];
        if (net->fp32)
          conv_f32(net, ti.act, l.Wt32, l.bias, to.act, B, Ho, Wo, l.cinp, l.coutp, op.relu, 0);
        else
          conv(net, ti.act, l.Wt, l.bias, to.act, B, Ho, Wo, l.cinp, l.coutp, op.relu, 0);
        break;
      }
      case kPool:
        k_pool2<<<row_grid(B * Ho, Wo, to.C), 256, 0, net->st>>>(ti.act, to.act, B * Ho, Ho, Wo, to.C);
        break;
      case kUp:
        k_up2<<<row_grid(B * Ho, Wo, to.C), 256, 0, net->st>>>(ti.act, to.act, B * Ho, Ho, Wo, to.C);
        break;
      case kAdd:
        k_add<<<blocks(n_out / 4), 256, 0, net->st>>>(reinterpret_cast<const float4*>(ti.act),
                                                        reinterpret_cast<const float4*>(net->T[op.in2].act),
                                                        reinterpret_cast<float4*>(to.act), n_out / 4);
        break;
    }
  }
  return launch_check(net, "forward");
}

// Reverse pass from the (padded) output gradient already in T[y_t].grad:
// fills every layer's dW / db and, when want_dx, T[x_t].grad.
lbm_status backward(nop_net* net, int B, bool want_dx) {
  const int H = net->cfg.height, W = net->cfg.width;
  for (size_t k = 0; k < net->T.size(); ++k) {
    if ((int)k == net->y_t) continue;
    const Tensor& t = net->T[k];
    NCK(cudaMemsetAsync(t.grad, 0, (size_t)pixels(net, t.level, B) * t.C * sizeof(float), net->st));
  }
  for (int i = (int)net->ops.size() - 1; i >= 0; --i) {
    const Op& op = net->ops[i];
    const Tensor& ti = net->T[op.in];
    const Tensor& to = net->T[op.out];
    const int Hi = H >> ti.level, Wi = W >> ti.level;
    const long long n_in = pixels(net, ti.level, B) * ti.C;
    switch (op.kind) {
      case kConv: {
        const Layer& l = net->L[op.layer];
        const long long P = pixels(net, to.level, B);
        if (op.relu)
          k_relu_mask<<<blocks(P * to.C / 4), 256, 0, net->st>>>(reinterpret_cast<const float4*>(to.act),
                                                                  reinterpret_cast<float4*>(to.grad), P * to.C / 4);
        const int nchunk = wgrad_chunks(B, Hi, Wi);
        if (net->fp32) {
          const long long P = (long long)B * Hi * Wi;
          const long long len = (long long)l.coutp * 9 * l.cinp;
          dim3 wg((unsigned)nchunk, (unsigned)((len + 127) / 128), 1u);
          k_conv3x3_wgrad_f32<<<wg, 128, 0, net->st>>>(to.grad, ti.act, net->part, B, Hi, Wi, l.cinp, l.coutp,
                                                        (P + nchunk - 1) / nchunk);
        } else if (Wi % kRowPx == 0 && l.coutp <= kWtM && l.coutp % 8 == 0 && l.cinp % 8 == 0) {
          // tensor cores: one CTA per (chunk, 32 input channels, row shift)
          dim3 wt((unsigned)nchunk * 3u * (unsigned)((l.cinp + kWtN - 1) / kWtN), 1u, 1u);
          k_conv3x3_wgrad_tc<<<wt, 128, kWtSmem, net->st>>>(to.grad, ti.act, net->part, B, Hi, Wi, l.cinp, l.coutp,
                                                            net->tc_status);
        } else {
          dim3 wg((unsigned)nchunk, (unsigned)((l.coutp + 31) / 32), (unsigned)((l.cinp + 31) / 32));
          k_conv3x3_wgrad<<<wg, 128, 0, net->st>>>(to.grad, ti.act, net->part, B, Hi, Wi, l.cinp, l.coutp);
        }
        const long long len = (long long)l.coutp * 9 * l.cinp;
        k_sum_chunks<<<(unsigned)((len + 31) / 32), dim3(32, 8), 0, net->st>>>(net->part, nchunk, len, l.dW);
        const int nbias = (int)((P + kWChunk - 1) / kWChunk);
        k_bias_partial<<<nbias, dim3(l.coutp, 4), 0, net->st>>>(to.grad, net->part, P, l.coutp);
        k_sum_chunks<<<(unsigned)((l.coutp + 31) / 32), dim3(32, 8), 0, net->st>>>(net->part, nbias, l.coutp, l.db);
        if (op.in != net->x_t || want_dx) {
          if (net->fp32)
            conv_f32(net, to.grad, l.Wf32, nullptr, ti.grad, B, Hi, Wi, l.coutp, l.cinp, 0, 1);
          else
            conv(net, to.grad, l.Wf, nullptr, ti.grad, B, Hi, Wi, l.coutp, l.cinp, 0, 1);
        }
        break;
      }
      case kPool:
        k_pool2_bwd<<<row_grid(B * Hi, Wi, ti.C), 256, 0, net->st>>>(to.grad, ti.grad, B * Hi, Hi, Wi, ti.C);
        break;
      case kUp:
        k_up2_bwd<<<row_grid(B * Hi, Wi, ti.C), 256, 0, net->st>>>(to.grad, ti.grad, B * Hi, Hi, Wi, ti.C);
        break;
      case kAdd: {
        const long long n = pixels(net, to.level, B) * to.C;
        k_acc<<<blocks(n / 4), 256, 0, net->st>>>(reinterpret_cast<const float4*>(to.grad),
                                                    reinterpret_cast<float4*>(ti.grad), n / 4);
        k_acc<<<blocks(n / 4), 256, 0, net->st>>>(reinterpret_cast<const float4*>(to.grad),
                                                    reinterpret_cast<float4*>(net->T[op.in2].grad), n / 4);
        break;
      }
    }
  }
  for (const Layer& l : net->L) {
    const long long n = (long long)l.cout * 9 * l.cin;
    k_unpad_grad<<<blocks(n), 256, 0, net->st>>>(l.dW, l.db, l.cin, l.cout, l.cinp, net->grad + l.offset);
  }
  return launch_check(net, "backward");
}

lbm_status check_batch(nop_net* net, int batch) {
  if (batch < 1 || batch > net->cfg.max_batch) return fail(net, LBM_EINVAL, "batch outside 1..max_batch");
  return LBM_OK;
}

lbm_status load_input(nop_net* net, int B, const float* x) {
  const Tensor& t = net->T[net->x_t];
  const long long P = pixels(net, 0, B);
  k_pad_channels<<<blocks(P * t.C), 256, 0, net->st>>>(x, t.act, P, net->cfg.in_channels, t.C);
  return launch_check(net, "k_pad_channels");
}

}  // namespace

extern "C" {

lbm_status nop_config_default(nop_config* cfg) {
  if (!cfg) return LBM_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->struct_size = sizeof(nop_config);
  cfg->height = 256;
  cfg->width = 512;
  cfg->max_batch = 8;
  cfg->in_channels = 3;
  cfg->out_channels = 4;
  cfg->channels[0] = 32;
  cfg->channels[1] = 64;
  cfg->channels[2] = 96;
  cfg->channels[3] = 128;
  return LBM_OK;
}

lbm_status nop_create(const nop_config* cfg, nop_net** out) {
  if (!cfg || !out || cfg->struct_size != sizeof(nop_config)) return LBM_EINVAL;
  *out = nullptr;
  if (cfg->height < 8 || cfg->width < 8 || cfg->height % 8 || cfg->width % 8 || cfg->max_batch < 1 ||
      cfg->in_channels < 1 || cfg->in_channels > 16 || cfg->out_channels < 1 || cfg->out_channels > 16)
    return LBM_EINVAL;
  for (int l = 0; l < 4; ++l)
    if (cfg->channels[l] < 16 || cfg->channels[l] > 256 || cfg->channels[l] % 16) return LBM_EINVAL;
  DeviceGuard dg(cfg->device);
  if (dg.status() != cudaSuccess) return LBM_ECUDA;
  nop_net* net = new nop_net();
  net->cfg = *cfg;
  if (cfg->stream) {
    net->st = static_cast<cudaStream_t>(cfg->stream);
  } else {
    if (cudaStreamCreateWithFlags(&net->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete net;
      return LBM_ECUDA;
    }
    net->own_stream = true;
  }
  build_graph(net);
  const int B = cfg->max_batch;
  lbm_status s = LBM_OK;
  for (Tensor& t : net->T) {
    const long long n = pixels(net, t.level, B) * t.C;
    if (!s) s = dalloc(net, &t.act, n);
    if (!s) s = dalloc(net, &t.grad, n);
  }
  const long long np = net->n_params;
  if (!s) s = dalloc(net, &net->master, np);
  if (!s) s = dalloc(net, &net->grad, np);
  if (!s) s = dalloc(net, &net->adam_m, np);
  if (!s) s = dalloc(net, &net->adam_v, np);
  for (const Op& op : net->ops) {
    if (op.kind != kConv) continue;
    const Layer& l = net->L[op.layer];
    const int lv = net->T[op.out].level;
    const long long nw = wgrad_chunks(B, cfg->height >> lv, cfg->width >> lv);
    const long long nb = (pixels(net, lv, B) + kWChunk - 1) / kWChunk;
    net->part_len = std::max(net->part_len, std::max(nw * l.coutp * 9 * l.cinp, nb * l.coutp));
  }
  for (Layer& l : net->L) {
    const long long n = (long long)l.coutp * 9 * l.cinp;
    if (!s) s = dalloc(net, &l.Wt, n);
    if (!s) s = dalloc(net, &l.Wf, n);
    if (!s) s = dalloc(net, &l.bias, l.coutp);
    if (!s) s = dalloc(net, &l.dW, n);
    if (!s) s = dalloc(net, &l.db, l.coutp);
  }
  if (!s) s = dalloc(net, &net->part, net->part_len);
  net->loss_blocks = (int)blocks(pixels(net, 0, B) * net->T[net->y_t].C);
  if (!s) s = dalloc(net, &net->loss_part, net->loss_blocks);
  if (!s) s = dalloc(net, &net->loss_dev, 1);
  if (!s) s = dalloc(net, &net->fields, 4 * (long long)cfg->height * cfg->width);
  if (!s) s = dalloc(net, &net->tc_status, 1);
  if (!s && cudaMemsetAsync(net->tc_status, 0, sizeof(int), net->st) != cudaSuccess) s = LBM_ECUDA;
  if (!s && (cudaMemsetAsync(net->master, 0, np * sizeof(float), net->st) != cudaSuccess ||
             cudaMemsetAsync(net->adam_m, 0, np * sizeof(float), net->st) != cudaSuccess ||
             cudaMemsetAsync(net->adam_v, 0, np * sizeof(float), net->st) != cudaSuccess ||
             cudaStreamSynchronize(net->st) != cudaSuccess))
    s = LBM_ECUDA;
  if (s) {
    nop_destroy(net);
    return s;
  }
  *out = net;
  return LBM_OK;
}

void nop_destroy(nop_net* net) {
  if (!net) return;
  DeviceGuard dg(net->cfg.device);
  if (net->st) cudaStreamSynchronize(net->st);
  for (void* p : net->allocs) cudaFree(p);
  if (net->own_stream && net->st) cudaStreamDestroy(net->st);
  delete net;
}

lbm_status nop_set_fp32(nop_net* net, int on) {
  if (!net) return LBM_EINVAL;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  if (on && !net->L.empty() && !net->L[0].Wt32) {
    for (Layer& l : net->L) {
      const long long n = (long long)l.coutp * 9 * l.cinp;
      lbm_status s = dalloc(net, &l.Wt32, n);
      if (!s) s = dalloc(net, &l.Wf32, n);
      if (s) return s;
    }
  }
  net->fp32 = on != 0;
  net->prepared = false;
  return LBM_OK;
}

const char* nop_last_error(const nop_net* net) { return net ? net->err.c_str() : "null network"; }

long long nop_param_count(const nop_net* net) { return net ? net->n_params : 0; }

lbm_status nop_init_params(nop_net* net, unsigned long long seed) {
  if (!net) return LBM_EINVAL;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  for (const Layer& l : net->L)
    k_init_layer<<<blocks(l.size()), 256, 0, net->st>>>(net->master + l.offset, l.cin, l.cout, seed, l.offset);
  NCK(cudaMemsetAsync(net->adam_m, 0, net->n_params * sizeof(float), net->st));
  NCK(cudaMemsetAsync(net->adam_v, 0, net->n_params * sizeof(float), net->st));
  net->adam_t = 0;
  net->prepared = false;
  NCK(cudaStreamSynchronize(net->st));
  return launch_check(net, "k_init_layer");
}

lbm_status nop_set_params(nop_net* net, int is_device, const float* params) {
  if (!net || !params) return LBM_EINVAL;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  NCK(cudaMemcpyAsync(net->master, params, net->n_params * sizeof(float),
                      is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, net->st));
  NCK(cudaMemsetAsync(net->adam_m, 0, net->n_params * sizeof(float), net->st));
  NCK(cudaMemsetAsync(net->adam_v, 0, net->n_params * sizeof(float), net->st));
  net->adam_t = 0;
  net->prepared = false;
  NCK(cudaStreamSynchronize(net->st));
  return LBM_OK;
}

lbm_status nop_get_params(const nop_net* cnet, int is_device, float* params) {
  nop_net* net = const_cast<nop_net*>(cnet);
  if (!net || !params) return LBM_EINVAL;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  NCK(cudaMemcpyAsync(params, net->master, net->n_params * sizeof(float),
                      is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, net->st));
  NCK(cudaStreamSynchronize(net->st));
  return LBM_OK;
}

lbm_status nop_forward(nop_net* net, int batch, const float* x, float* y) {
  if (!net || !x || !y) return LBM_EINVAL;
  lbm_status s = check_batch(net, batch);
  if (s) return s;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  if ((s = load_input(net, batch, x)) || (s = forward(net, batch))) return s;
  const Tensor& t = net->T[net->y_t];
  const long long P = pixels(net, 0, batch);
  k_crop_channels<<<blocks(P * net->cfg.out_channels), 256, 0, net->st>>>(t.act, y, P, t.C, net->cfg.out_channels);
  NCK(cudaStreamSynchronize(net->st));
  return finish(net, "nop_forward");
}

lbm_status nop_backward(nop_net* net, int batch, const float* x, const float* dy, float* dparams, float* dx) {
  if (!net || !x || !dy) return LBM_EINVAL;
  lbm_status s = check_batch(net, batch);
  if (s) return s;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  if ((s = load_input(net, batch, x)) || (s = forward(net, batch))) return s;
  const Tensor& t = net->T[net->y_t];
  const long long P = pixels(net, 0, batch);
  k_pad_channels<<<blocks(P * t.C), 256, 0, net->st>>>(dy, t.grad, P, net->cfg.out_channels, t.C);
  if ((s = backward(net, batch, dx != nullptr))) return s;
  if (dparams)
    NCK(cudaMemcpyAsync(dparams, net->grad, net->n_params * sizeof(float), cudaMemcpyDeviceToDevice, net->st));
  if (dx) {
    const Tensor& tx = net->T[net->x_t];
    k_crop_channels<<<blocks(P * net->cfg.in_channels), 256, 0, net->st>>>(tx.grad, dx, P, tx.C,
                                                                          net->cfg.in_channels);
  }
  NCK(cudaStreamSynchronize(net->st));
  return finish(net, "nop_backward");
}

lbm_status nop_train_step(nop_net* net, int batch, const float* x, const float* target, float lr, double* loss) {
  if (!net || !x || !target || !(lr >= 0.f)) return LBM_EINVAL;
  lbm_status s = check_batch(net, batch);
  if (s) return s;
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  if ((s = load_input(net, batch, x)) || (s = forward(net, batch))) return s;
  const Tensor& t = net->T[net->y_t];
  const long long P = pixels(net, 0, batch);
  const double inv_count = 1.0 / ((double)P * net->cfg.out_channels);
  const int nb = (int)blocks(P * t.C);
  k_mse<<<nb, 256, 0, net->st>>>(t.act, target, t.grad, net->loss_part, P, t.C, net->cfg.out_channels, inv_count);
  k_mse_total<<<1, 1024, 0, net->st>>>(net->loss_part, nb, inv_count, net->loss_dev);
  if ((s = backward(net, batch, false))) return s;
  net->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)net->adam_t));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)net->adam_t));
  k_adam<<<blocks(net->n_params), 256, 0, net->st>>>(net->master, net->grad, net->adam_m, net->adam_v, net->n_params,
                                                      lr, b1, b2, 1e-8f, c1, c2);
  net->prepared = false;
  double l = 0.0;
  NCK(cudaMemcpyAsync(&l, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, net->st));
  NCK(cudaStreamSynchronize(net->st));
  if (loss) *loss = l;
  return finish(net, "nop_train_step");
}

lbm_status nop_infer_into(nop_net* net, lbm_handle* h, const float* x, const double off[4], const double scale[4]) {
  if (!net || !h || !x || !off || !scale) return LBM_EINVAL;
  if (h->D != 2 || h->g.n[0] != net->cfg.width || h->g.n[1] != net->cfg.height || net->cfg.out_channels != 4)
    return fail(net, LBM_EINVAL, "solver must be D2Q9 of the network's grid, network with 4 outputs");
  DeviceGuard dg(net->cfg.device);
  NCK(dg.status());
  lbm_status s;
  if ((s = load_input(net, 1, x)) || (s = forward(net, 1))) return s;
  const long long N = (long long)net->cfg.height * net->cfg.width;
  double* rho = net->fields;
  double* u = rho + N;
  double* T = u + 2 * N;
  k_to_fields<<<blocks(N), 256, 0, net->st>>>(net->T[net->y_t].act, net->T[net->y_t].C, N, off[0], off[1], off[2],
                                              off[3], scale[0], scale[1], scale[2], scale[3], rho, u, T);
  NCK(cudaStreamSynchronize(net->st));
  if ((s = finish(net, "k_to_fields"))) return s;
  s = lbm_set_fields(h, 1, rho, u, T);
  if (s) return fail(net, s, "lbm_set_fields failed");
  return LBM_OK;
}

}  // extern "C"

__kernel void relu(__global int *data)
{
    int var0;
    var0 = data[get_global_id(0)];
    data[get_global_id(0)] = ((var0 < 0) ? 0 : var0);
}
